/*
 * swept2d.h -- C ABI of the two-dimensional swept solver (2D FTCS heat).
 *
 * The paper (Magee & Niemeyer, "An initial investigation of the performance of
 * GPU-based swept time-space decomposition") decomposes 1D problems and names
 * two dimensions as future work (Section "Conclusion").  This interface is that
 * extension for the 2D heat equation on square cells,
 *   T'_{i,j} = Fo (T_{i-1,j} + T_{i+1,j} + T_{i,j-1} + T_{i,j+1}) + (1 - 4 Fo) T_{i,j},
 *   Fo = alpha dt / dx^2,
 * the 2D form of Eq. HeatDisc, on an nx x ny grid, periodic or insulated.  As in 1D, the
 * swept decomposition does not change the scheme: swept2d_step_n and
 * classic2d_step_n produce the same values bit for bit.
 *
 * Status codes, dtypes and boundary codes are those of swept.h.
 *
 * Layout: the state is nx * ny contiguous values of the handle's dtype,
 * row-major with x fastest: u[j * nx + i].  The caller owns the state and the
 * workspace (device memory); the library never allocates device memory.  The
 * handle owns host memory, a private capture stream and cached CUDA graphs.
 * Every compute call is asynchronous on the caller's stream and returns a
 * status; nothing throws across the ABI.  swept2d_last_error describes the
 * last failure of a handle.  A handle is not thread-safe: calls on one handle
 * must not overlap.
 */
#ifndef SWEPT2D_H
#define SWEPT2D_H

#include <stddef.h>
#include <stdint.h>

#include "swept.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Problem and launch configuration.
 *   dtype    SWEPT_F32 or SWEPT_F64
 *   bc       SWEPT_BC_PERIODIC, or SWEPT_BC_REFLECTIVE: insulated ends, mirror
 *            walls at -1/2 and n - 1/2 on both axes (cell -1 reads cell 0, cell n
 *            reads cell n - 1)
 *   nx, ny   grid points along x and y: multiples of tile_w, at least two tiles
 *            per axis, ny <= 65535
 *   dx, dt   grid spacing (both axes) and timestep; alpha the diffusivity.
 *            Stability (Fo <= 1/4) is the caller's responsibility.
 *   tile_w   W: the tile is W x W points, W a multiple of 4 (so that the half
 *            cycle h = W / 2 is even), 8 <= W <= 64 for FP64 and <= 128 for
 *            FP32 (two (W + 2)^2 level rows in shared memory); 0 = library choice
 *   threads  threads per block, a multiple of 32, <= 1024; 0 = 256
 *   persistent  0: one launch per pass (pyramid, then a bridge launch and an
 *            octahedron launch per half cycle); 1: one persistent launch whose
 *            resident blocks run the same pieces from a queue in launch order,
 *            each piece waiting only for the counters of the pieces its inputs
 *            come from (tiles / bridges of the previous stage), so successive
 *            half cycles overlap.  Same values bit for bit.
 *   reserved must be zero.
 */
typedef struct {
  int32_t dtype;
  int32_t bc;
  int64_t nx;
  int64_t ny;
  double dx;
  double dt;
  double alpha;
  int32_t tile_w;
  int32_t threads;
  int32_t persistent;
  int32_t reserved[3];
} swept2d_config;

typedef struct {
  int32_t tile_w;          /* W */
  int32_t threads;         /* threads per block */
  int32_t half_cycle;      /* h = W / 2: levels per half cycle */
  int32_t persistent;      /* 1 for the persistent queue kernel */
  int64_t tiles_x, tiles_y;
  int64_t smem_bytes;      /* dynamic shared memory per block */
  int64_t workspace_bytes; /* same as swept2d_workspace_size() */
} swept2d_plan_info;

typedef struct swept2d_handle swept2d_handle;

/* Validate `cfg`, choose the plan and create a handle (host memory only).
 * SWEPT_EINVAL for an invalid configuration (*out is then NULL). */
swept_status swept2d_init(const swept2d_config* cfg, swept2d_handle** out);

/* Bytes of device workspace the handle needs: two strip buffers (2 W^2 + 4 W
 * values per tile each: the pyramids' side strips of every level), one band
 * buffer (2 W^2 - 4 W values per tile: the end bands of its two bridges; two
 * for a persistent handle), the classic path's second state array, a status
 * word and, for a persistent handle, 3 counters per tile and the queue. */
swept_status swept2d_workspace_size(const swept2d_handle* h, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, at least
 * swept2d_workspace_size bytes) as the workspace.  Drops cached graphs. */
swept_status swept2d_bind_workspace(swept2d_handle* h, void* ws_dev, size_t bytes);

/* Advance u_dev (device, nx * ny values, in place) by nsteps timesteps with the
 * 2D swept decomposition: per half cycle of h = W / 2 steps one bridge launch
 * and one octahedron launch (captured in CUDA graphs), or the single persistent
 * launch; the state read and written once per call.  nsteps = 0 is a no-op.
 * A persistent wait that runs out (SWEPT_OPT_SPIN_LIMIT polls) stops the
 * kernel and latches SWEPT_ETIMEOUT into the status word (swept2d_sync_status);
 * the state is then undefined. */
swept_status swept2d_step_n(swept2d_handle* h, void* u_dev, int64_t nsteps, void* stream);

/* The same advance with one launch per timestep (global memory in and out):
 * the baseline the swept decomposition is compared with.  Bit-identical. */
swept_status classic2d_step_n(swept2d_handle* h, void* u_dev, int64_t nsteps, void* stream);

swept_status swept2d_get_plan(const swept2d_handle* h, swept2d_plan_info* out);

/* Options (drop cached graphs):
 *   SWEPT_OPT_SPIN_LIMIT  polls before a persistent wait gives up (default 2^24)
 *   SWEPT_OPT_START_ITEM  first queue item the persistent kernel claims
 *                         (default 0; > 0 skips items, so the waits for them
 *                         run out: used to exercise the timeout path)
 *   SWEPT2D_OPT_CHECK_DROP_WAIT  swept2d_check_schedule only: drop the last
 *                         wait of this queue item (-1: none, the default), to
 *                         show that the replay finds the race this opens
 * SWEPT_EINVAL for an unknown option or a value out of range. */
enum { SWEPT2D_OPT_CHECK_DROP_WAIT = 16 };
swept_status swept2d_set_option(swept2d_handle* h, int32_t option, int64_t value);

/* Wait for the stream, read and clear the status word: SWEPT_OK, or
 * SWEPT_ETIMEOUT if a persistent wait ran out since the last call. */
swept_status swept2d_sync_status(swept2d_handle* h, void* stream);

/* Host-only symbolic replay of the 2D launch sequence for nsteps steps (no GPU):
 * checks that every point of every level is computed exactly once, only after
 * its five stencil inputs hold the previous level, that no two blocks of one
 * launch touch a location one of them writes, and that the final state holds
 * level nsteps everywhere.  For a persistent handle it replays the queue in
 * order instead, and checks that every item waits only for earlier items, that
 * counters only grow, and that every access to a location follows (through
 * the waits' transitive closure) the last write of it, and every write the
 * reads of the value it replaces (at most 16384 items, else SWEPT_EINVAL).
 * *computed receives the number of point updates.
 * SWEPT_EDEVICE with a message in swept2d_last_error if a check fails. */
swept_status swept2d_check_schedule(swept2d_handle* h, int64_t nsteps, int64_t* computed);

/* Copy the last error message of the handle into buf (always terminated). */
swept_status swept2d_last_error(const swept2d_handle* h, char* buf, size_t len);

void swept2d_free(swept2d_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SWEPT2D_H */
