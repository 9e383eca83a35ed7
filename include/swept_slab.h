/*
 * swept_slab.h - one grid split over several ranks (one GPU each) for the
 * swept decomposition (libswept.so).
 *
 * The paper names a multi-GPU swept solver as future work: the swept rule
 * needs communication only at the triangle edges, so GPUs that each hold part
 * of the grid trade only those edges (Section "Conclusion"; the exchange of
 * Section "First-order", Fig. collection).  This API runs that solver one rank
 * at a time: the caller owns the transport between ranks (NCCL, MPI, a copy),
 * and the library says what to launch and what to trade.
 *
 * Partition.  The grid's nt = floor(n / tile_w) tiles are split into nranks
 * contiguous slabs, as evenly as possible; rank r runs blocks [b0, b0 + nb) of
 * every swept pass (up, diamond, down and remainder passes alike).  The ranks
 * form a ring (rank 0's left neighbour is rank nranks - 1) for both boundary
 * conditions.  Each rank advances exactly the points and sub-timesteps that
 * blocks [b0, b0 + nb) advance on one GPU, in the same operation order, so the
 * gathered result equals swept_step_n (and classic_step_n) bit for bit.
 *
 * Per rank (all device memory caller-owned):
 *   - a state array of state_len values per component holding global points
 *     [x0, x0 + state_len), component c at offset c * state_len, no wrap
 *     (layout as swept.h otherwise: Euler is rho | m | E).  On entry and on
 *     exit of a solve the rank's points are [x0, x1); the W/2 values past x1
 *     are scratch that the odd passes write;
 *   - a workspace of workspace_bytes holding two edge buffers (e0, e1) of
 *     edge_values values each, at the value offsets e0_offset / e1_offset.
 *
 * A solve of nsteps timesteps is swept_slab_launch_count() launches.  After
 * launch i (and before launch i + 1) each rank posts the transfers that
 * swept_slab_xfers(i) lists: half an edge block (2 r h C values) before every
 * diamond pass, and after an odd down pass or the remainder's gap pass the
 * values its blocks wrote past x1.  A rank's k-th send to one side matches that
 * neighbour's k-th receive from the other side, in posting order; post them
 * together (e.g. one grouped send/receive) so that no rank waits on a send
 * before posting its receive.  With nranks = 1 the sends go to the rank itself.
 * Transfers must complete, on the launching stream's order, before the next
 * launch reads them.
 *
 * Limits: nranks <= nt; per-pass launches only (the config's persistent and
 * cluster must be 0); the plan (tile, threads, chunk, warp_tiles) is chosen as
 * by swept_init.  Every call returns a swept_status and never throws.
 */
#ifndef SWEPT_SLAB_H
#define SWEPT_SLAB_H

#include <stddef.h>
#include <stdint.h>

#include "swept.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swept_slab swept_slab;

/* What one rank holds (swept_slab_get_layout). */
typedef struct {
  int64_t first_block;     /* b0: the slab's first tile */
  int64_t blocks;          /* nb: tiles of the slab (>= 1) */
  int64_t x0, x1;          /* global points [x0, x1) the rank owns before and after a solve */
  int64_t state_len;       /* values per component of the state array (global points x0 .. x0 + state_len) */
  int64_t edge_values;     /* values of each edge buffer */
  int64_t e0_offset;       /* value offset of edge buffer 0 in the workspace */
  int64_t e1_offset;       /* value offset of edge buffer 1 in the workspace */
  int64_t workspace_bytes; /* bytes the rank's workspace must hold */
  int32_t tile_w, threads, half_cycle, value_bytes;
} swept_slab_layout;

/* One transfer between neighbouring ranks. */
typedef struct {
  int32_t peer;    /* -1: left neighbour (rank - 1 mod nranks); +1: right neighbour */
  int32_t recv;    /* 0: send these values; 1: receive into them */
  int32_t region;  /* 0: edge buffer 0; 1: edge buffer 1; 2: the state array */
  int32_t reserved;
  int64_t offset;  /* first value (of the handle's dtype) within that region */
  int64_t count;   /* values */
} swept_slab_xfer;

/* Rank `rank` (0 <= rank < nranks) of a grid split over nranks ranks.  cfg as
 * for swept_init; the plan is the one swept_init would choose.  Uses the
 * current CUDA device (as swept_init does; without one only the host calls work).
 * Errors: SWEPT_EINVAL (bad config, rank, or nranks > tiles), SWEPT_EUNSUPPORTED
 * (persistent or cluster requested, or a grid too small for two tiles). */
swept_status swept_slab_init(const swept_config* cfg, int32_t rank, int32_t nranks, swept_slab** out);

swept_status swept_slab_get_layout(const swept_slab* h, swept_slab_layout* out);

/* Bind the rank's workspace (>= workspace_bytes, 256-byte aligned device memory). */
swept_status swept_slab_bind_workspace(swept_slab* h, void* ws_dev, size_t bytes);

/* Launches of a solve of nsteps timesteps (0 for nsteps = 0). */
swept_status swept_slab_launch_count(const swept_slab* h, int64_t nsteps, int64_t* count);

/* Issue launch i (0 <= i < count) of a solve of nsteps timesteps on `stream`
 * over the rank's state array u_dev.  Asynchronous. */
swept_status swept_slab_launch(swept_slab* h, void* u_dev, int64_t nsteps, int64_t i, void* stream);

/* The transfers due after launch i of a solve of nsteps timesteps, in posting
 * order: up to `cap` entries into out[], their number into *n (at most 8). */
swept_status swept_slab_xfers(const swept_slab* h, int64_t nsteps, int64_t i, swept_slab_xfer* out, int32_t cap,
                              int32_t* n);

swept_status swept_slab_last_error(const swept_slab* h, char* buf, size_t len);
void swept_slab_free(swept_slab* h);

/* Host-only check of the partition: replays a solve of nsteps timesteps over
 * all nranks ranks symbolically (values replaced by (point, sub-timestep)
 * tags, the same pass phases and transfer lists the GPU path uses) and checks
 * that every stencil input holds the right point at the right sub-timestep,
 * that every (point, sub-timestep) is computed exactly once over all ranks, and
 * that each rank ends holding sub-timestep n_sub on [x0, x1).  *computed gets
 * the number of point-updates.  On failure returns SWEPT_EDEVICE with the
 * first violation in msg.  Limited to (nsteps S + 1) n <= 4e8 and
 * (nsteps S + 1) n nranks <= 2e9. */
swept_status swept_slab_check(const swept_config* cfg, int32_t nranks, int64_t nsteps, int64_t* computed, char* msg,
                              size_t len);

/* The symbolic replay of one rank, for checking a transport between processes
 * on the host: its buffers hold tags (two int64 per value: point, sub-timestep)
 * laid out as the rank's state array and edge buffers, so that a transport
 * can move them with the offsets and counts of swept_slab_xfers (x 2 int64).
 *   swept_slab_sym_buffer: region 0 / 1 / 2 as swept_slab_xfer; *tags points
 *       to 2 * (*values) int64 owned by the replay
 *   swept_slab_sym_launch: replay launch i (checks every stencil input)
 *   swept_slab_sym_finish: checks [x0, x1) holds sub-timestep n_sub and adds
 *       the rank's count of each (sub-timestep, point) update into counts
 *       ((nsteps S + 1) * n int32, caller-owned; over all ranks every entry of
 *       sub-timestep >= 1 must sum to 1).  SWEPT_EDEVICE + msg on a violation. */
typedef struct swept_slab_sym swept_slab_sym;
swept_status swept_slab_sym_init(const swept_config* cfg, int32_t rank, int32_t nranks, int64_t nsteps,
                                 swept_slab_sym** out);
swept_status swept_slab_sym_buffer(swept_slab_sym* s, int32_t region, int64_t** tags, int64_t* values);
swept_status swept_slab_sym_launch(swept_slab_sym* s, int64_t i, char* msg, size_t len);
swept_status swept_slab_sym_finish(swept_slab_sym* s, int32_t* counts, char* msg, size_t len);
void swept_slab_sym_free(swept_slab_sym* s);

#ifdef __cplusplus
}
#endif

#endif /* SWEPT_SLAB_H */
