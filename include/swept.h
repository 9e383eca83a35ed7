/*
 * swept.h - C ABI of the GB300 swept time-space decomposition library (libswept.so).
 *
 * Method: Magee & Niemeyer, "An initial investigation of the performance of
 * GPU-based swept time-space decomposition" (arXiv:1612.02495).
 *   - Problem statement: an explicit 1D stencil scheme on n grid points with a
 *     boundary condition, advanced a number of timesteps (Section "Test cases",
 *     Eq. HeatDisc, Eq. KSDisc, Appendix).
 *   - Swept rule: each thread block keeps a tile ("node") in shared memory,
 *     advances it as a shrinking triangle, passes only the triangle edges, then
 *     completes diamonds, zig-zagging the tiles by half a tile each pass
 *     (Section "First-order", Figs. firstorder and collection; Section
 *     "Second-order extended stencil", Fig. secondordersolution).
 *   - Classic decomposition: one kernel per sub-timestep through global memory
 *     (Section "Classic scheme", Fig. ClassicCode).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never allocates device memory (no cudaMalloc) and never frees
 *     caller memory.  Pointers named *_host are host pointers owned by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream are asynchronous on it unless stated otherwise.
 *   - Every call returns a swept_status and never throws.  On failure the
 *     handle (if any) keeps a message readable with swept_last_error().
 *   - Device-side errors (a bounded wait that ran out, a failed consistency
 *     check inside a kernel) are latched in a word of the bound workspace and
 *     returned by swept_sync_status().
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 *
 * State layout in device memory (dtype fixed per handle, contiguous):
 *   SWEPT_HEAT, SWEPT_KS : n values u[0..n)
 *   SWEPT_EULER          : 3*n values, structure of arrays (rho[0..n) | m[0..n) | E[0..n))
 */
#ifndef SWEPT_H
#define SWEPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SWEPT_OK = 0,
  SWEPT_EINVAL = 1,            /* bad argument or configuration */
  SWEPT_ENOMEM_WORKSPACE = 2,  /* bound workspace smaller than swept_workspace_size() */
  SWEPT_ECUDA = 3,             /* a CUDA runtime call failed (message in swept_last_error) */
  SWEPT_ETIMEOUT = 4,          /* a bounded device-side wait ran out */
  SWEPT_EUNSUPPORTED = 5,      /* valid request this build does not implement */
  SWEPT_ENOWORKSPACE = 6,      /* no workspace bound yet */
  SWEPT_EDEVICE = 7            /* a kernel's own consistency check failed */
} swept_status;

typedef enum {
  SWEPT_HEAT = 0,  /* u_t = alpha u_xx, FTCS (Eq. HeatDisc): r=1, one stage */
  SWEPT_KS = 1,    /* u_t = -u u_x - u_xx - nu u_xxxx, Eq. KSDisc + midpoint RK2 (Appendix): r=2, two stages */
  SWEPT_EULER = 2  /* 1D Euler, MUSCL-minmod + Rusanov + SSP-RK2 (not in the paper): r=2, two stages */
} swept_scheme;

typedef enum { SWEPT_F32 = 0, SWEPT_F64 = 1 } swept_dtype;

typedef enum {
  SWEPT_BC_PERIODIC = 0,   /* index i+k taken mod n (Appendix) */
  SWEPT_BC_REFLECTIVE = 1  /* mirror walls at x = -1/2 and n - 1/2: insulated ends for heat,
                              reflective walls (momentum negated) for Euler; not for KS */
} swept_bc;

/*
 * Problem and launch configuration.
 *   n        grid points, any n >= 2r + 1 (r = 1 heat, 2 KS/Euler): the paper's
 *            problem is a grid of n points, a stencil, a step count and a
 *            boundary condition (Section "Test cases", Eq. HeatDisc, Eq. KSDisc).
 *            The swept tiling takes floor(n / tile_w) >= 2 tiles; when tile_w
 *            does not divide n, the last tile is wider by X = n mod tile_w
 *            points (an up-trapezoid whose flat top of X points is handed from
 *            pass to pass), so every diamond keeps height h.  A grid with no
 *            legal tiling (n < 8r with tile_w = 0) still gets a handle, on which
 *            classic_step_n runs and the swept calls return SWEPT_EUNSUPPORTED.
 *   dx, dt   grid spacing and timestep
 *   param[0] heat: alpha (diffusivity); KS: nu (factor on u_xxxx, 1 = the
 *            paper's equation); Euler: gamma
 *   tile_w   points per tile W (the paper's node size / threads per block);
 *            0 = chosen by the library (a divisor of n when one gives enough
 *            tiles).  Must be a multiple of 4*r (r = 1 heat, 2 KS/Euler), so
 *            that the half-cycle h = W/(2r) is even, with n >= 2 W.  The cluster
 *            and warp_tiles modes need W to divide n.
 *   threads  threads per block, 0 = chosen by the library (<= 1024, multiple of 32)
 *   chunk    heat and KS: 1 = one point per thread per trip through a tier
 *            (strided; in FP32, radius-2 tiers take aligned pairs of points,
 *            the default); 2 = two strided points (j, j + threads) with both
 *            windows loaded first.  Euler: 1 = one thread per face in the flux
 *            phase of a tier; 2 = two threads per face (one per reconstructed
 *            side, exchanged by warp shuffle)
 *   persistent 0: one kernel launch per swept pass (graph-captured); 1: the
 *            passes form one queue of (pass, tile) items run by a persistent
 *            kernel whose blocks wait (bounded) only for the two tiles they read,
 *            so no block waits for a whole pass to finish
 *   cluster  1: (n / tile_w <= 16) one launch whose blocks form a single
 *            thread-block cluster; each block keeps its tile in shared memory
 *            for the whole solve and reads its neighbour's edges through
 *            distributed shared memory, with a cluster barrier between passes
 *   warp_tiles 1: heat and KS with tile_w = 32 P, P in {1, 2, 4, 8}: each
 *            tile is one warp (threads must be 0 or 32) whose lane l keeps
 *            points l P .. l P + P - 1 of the tier rows in registers and reads
 *            its stencil neighbours from the lanes beside it (up to ceil(r / P)
 *            lanes away; KS with P = 1 is the paper's 32-point register node,
 *            Section "Conclusion") by warp shuffle, so a tier needs no
 *            shared-memory access and no barrier.
 *            Works with the per-pass, persistent and cluster modes; results are
 *            bit-identical to the shared-memory tiers.
 * Stability (Fo <= 1/2, CFL) is the caller's responsibility and is not checked.
 */
typedef struct {
  int32_t scheme;   /* swept_scheme */
  int32_t dtype;    /* swept_dtype */
  int32_t bc;       /* swept_bc */
  int32_t reserved0;
  int64_t n;
  double dx;
  double dt;
  double param[4];
  int32_t tile_w;
  int32_t threads;
  int32_t chunk;    /* heat/KS: 1, or 2 (two strided points a trip); Euler: threads per face, 1 or 2; 0 = 1 */
  int32_t persistent; /* 1: swept_step_n runs all passes in one persistent kernel */
  int32_t cluster;    /* 1: the whole grid (2..16 tiles) is one thread-block cluster */
  int32_t warp_tiles; /* 1: one warp per tile, tier rows in registers, neighbours by warp shuffle */
  int32_t reserved[2];
} swept_config;

/* Plan chosen by swept_init (read-only report). */
typedef struct {
  int32_t tile_w;          /* W */
  int32_t threads;         /* threads per block */
  int32_t half_cycle;      /* h = W / (2r): sub-timesteps advanced per swept pass */
  int32_t radius;          /* r: stencil radius of one sub-timestep */
  int32_t stages;          /* S: sub-timesteps per timestep */
  int32_t components;      /* C: values per grid point */
  int64_t tiles;           /* n / W */
  int64_t smem_bytes;      /* dynamic shared memory per block of the swept kernels */
  int64_t workspace_bytes; /* same as swept_workspace_size() */
  int32_t chunk;           /* points per thread per tier */
  int32_t persistent;      /* 1: persistent kernel */
  int32_t cluster;         /* 1: single-cluster kernel */
  int32_t warp_tiles;      /* 1: tier rows in registers, one warp per tile */
  int32_t last_tile_extra; /* X = n - tiles * W: extra points of the last tile (0 when W divides n) */
} swept_plan_info;

typedef struct swept_handle swept_handle;

/* Validate `cfg`, choose the plan and create a handle (host memory only).
 * Errors: SWEPT_EINVAL (bad cfg, NULL pointers), SWEPT_ECUDA (no device). */
swept_status swept_init(const swept_config* cfg, swept_handle** out);

/* Bytes of device workspace the handle needs: the ping-pong edge buffers of
 * the swept passes (Section "First-order": the global "left"/"right" arrays),
 * the classic path's intermediate stage array, and a status word. */
swept_status swept_workspace_size(const swept_handle* h, size_t* bytes);

/* Bind caller-owned device workspace (>= swept_workspace_size bytes, 256-byte
 * aligned).  Rebinding drops cached CUDA graphs.  Errors: SWEPT_EINVAL,
 * SWEPT_ENOMEM_WORKSPACE. */
swept_status swept_bind_workspace(swept_handle* h, void* ws_dev, size_t bytes);

/* Advance u_dev (layout above) by nsteps full timesteps in place with the swept
 * rule: up-triangle, diamonds, down-triangle, then a trapezoid pair for the
 * sub-timesteps left over (nsteps * S mod h).  nsteps == 0 is a no-op.
 * Results equal classic_step_n bit for bit (same per-point operation order).
 * Errors: SWEPT_EINVAL, SWEPT_ENOWORKSPACE, SWEPT_ECUDA. */
swept_status swept_step_n(swept_handle* h, void* u_dev, int64_t nsteps, void* stream);

/* Same advance with the classic decomposition: one kernel per sub-timestep
 * (Fig. ClassicCode), captured into CUDA graphs. */
swept_status classic_step_n(swept_handle* h, void* u_dev, int64_t nsteps, void* stream);

/* End-to-end call for callers holding host data: copies u_host_in (layout
 * above) to u_dev, advances nsteps (swept if use_swept != 0, else classic),
 * copies the result to u_host_out, and synchronizes `stream` before returning.
 * u_host_in may equal u_host_out.  Pinned host memory gives asynchronous copies. */
swept_status swept_run_host(swept_handle* h, const void* u_host_in, void* u_host_out, void* u_dev, int64_t nsteps,
                            int32_t use_swept, void* stream);

/* Discrete adjoint of swept_step_n for SWEPT_KS and SWEPT_HEAT in SWEPT_F64
 * (not in the paper).  The loss L depends on u(T), the state after nsteps
 * steps from u0; given gT_dev = dL/du(T) it writes g_u0_dev = dL/du0 (layout of
 * u) and g_param_dev[0] = dL/dparam[0] (nu for KS, alpha for heat), one double.
 * The reverse sweep runs the swept schedule backwards with the transposed
 * stencil (same radius and tiers); each tier reads the forward state of its
 * sub-timestep from a tape.  Forward states are recomputed segment by segment
 * from checkpoints in ckpt_dev: u at the start of every segment of K steps,
 * plus one segment's tape of S*K + 1 tiers.  K is the largest whole number of
 * passes (h/S steps) whose layout fits ckpt_bytes; ckpt_bytes =
 * swept_adjoint_ckpt_size() is the smallest layout (K near sqrt(nsteps / S)
 * rounded to whole passes: about 2 sqrt(S nsteps) + h copies of the state),
 * and a buffer large enough for K = nsteps stores the whole run and
 * recomputes nothing.  Any K recomputes each step at most once.
 * If u0_dev is NULL, the checkpoints and the last segment's tape written by the
 * most recent swept_forward_ckpt on this handle (same ckpt_dev, ckpt_bytes,
 * nsteps) are used, so only the earlier segments are recomputed; otherwise the
 * checkpointing forward pass from u0_dev runs first.  g_u0_dev may alias
 * gT_dev.  Errors: SWEPT_EUNSUPPORTED (scheme/dtype), SWEPT_EINVAL (no
 * matching forward for u0_dev = NULL), SWEPT_ENOMEM_WORKSPACE (ckpt too small). */
swept_status swept_adjoint_ckpt_size(const swept_handle* h, int64_t nsteps, size_t* bytes);
swept_status swept_forward_ckpt(swept_handle* h, void* u_dev, int64_t nsteps, void* ckpt_dev, size_t ckpt_bytes,
                                void* stream);
swept_status swept_adjoint(swept_handle* h, const void* u0_dev, const void* gT_dev, int64_t nsteps, void* g_u0_dev,
                           void* g_param_dev, void* ckpt_dev, size_t ckpt_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Batched solves (not in the paper): many independent heat / KS problems of   */
/* different sizes and step counts, all in one dtype, advanced by one          */
/* persistent kernel launch (captured in a CUDA graph).  Each problem runs the */
/* same swept launch sequence as swept_step_n (results equal it bit for bit);  */
/* the passes of all problems form one work queue of (problem, pass, tile)     */
/* items ordered by pass, whose blocks wait (bounded) for the two tiles they   */
/* read to finish the previous pass.                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t scheme;  /* SWEPT_HEAT or SWEPT_KS (periodic) */
  int32_t tile_w;  /* W for this problem, 0 = largest power of two <= 512 giving >= 2 tiles */
  int64_t n;       /* grid points (a multiple of W, >= 2W) */
  int64_t nsteps;  /* timesteps */
  double dx, dt;
  double param;    /* alpha (heat) or nu (KS) */
} swept_batch_problem;

typedef struct swept_batch swept_batch;

enum {
  SWEPT_BATCH_SPIN_LIMIT = 1, /* iterations a block waits for an input tile before SWEPT_ETIMEOUT (default 2^24) */
  SWEPT_BATCH_START_ITEM = 2, /* first queue item to run (0; larger values leave inputs missing: for fault tests) */
  SWEPT_BATCH_GRID = 3        /* cap on the persistent grid (0 = all co-resident blocks) */
};

/* Plan a batch (host only).  threads = block size for every item (0 = 256).
 * Errors: SWEPT_EINVAL (a problem violates the constraints above). */
swept_status swept_batch_plan(const swept_batch_problem* problems, int64_t count, int32_t dtype, int32_t threads,
                              swept_batch** out);
/* Layout: offsets[count] = first value of each problem's state in the batch
 * state array (256-byte aligned starts), state_values = its length, ws_bytes =
 * device workspace size, items = queue length.  Any output may be NULL. */
swept_status swept_batch_sizes(const swept_batch* b, int64_t* offsets, int64_t* state_values, size_t* ws_bytes,
                               int64_t* items);
/* Bind caller-owned workspace (uploads the plan; synchronous). */
swept_status swept_batch_bind_workspace(swept_batch* b, void* ws_dev, size_t bytes);
swept_status swept_batch_set_option(swept_batch* b, int32_t option, int64_t value);
/* Advance every problem of the batch state u_dev by its nsteps, in place. */
swept_status swept_batch_run(swept_batch* b, void* u_dev, void* stream);
/* The same advance with the classic decomposition (Section "Classic scheme",
 * Fig. ClassicCode), the baseline of swept_batch_run: launch k advances every
 * problem that still has a sub-timestep k by one sub-timestep through global
 * memory, one point per thread, with classic_step_n's per-point operation
 * (results equal swept_batch_run bit for bit).  The launches are captured into
 * CUDA graphs of 1024 launches, cached per u_dev.  It uses the tmp area of the
 * bound workspace (one value per state value). */
swept_status swept_batch_run_classic(swept_batch* b, void* u_dev, void* stream);
/* Synchronize `stream`, then return SWEPT_ETIMEOUT if a bounded wait ran out. */
swept_status swept_batch_sync_status(swept_batch* b, void* stream);
swept_status swept_batch_last_error(const swept_batch* b, char* buf, size_t len);
void swept_batch_free(swept_batch* b);

/* Tracing: run swept_step_n's launch sequence for nsteps on `stream` with
 * direct launches (no graph) and a CUDA event pair around every launch, then
 * synchronize.  out_ms[4] receives the summed device time and out_count[4] the
 * number of launches of each kind: [0] up-triangle, [1] diamond, [2]
 * down-triangle, [3] remainder pair.  u_dev is advanced exactly as by
 * swept_step_n. */
swept_status swept_profile_passes(swept_handle* h, void* u_dev, int64_t nsteps, void* stream, double* out_ms,
                                  int64_t* out_count);

/* Size in bytes of the device array swept_step_n_static keeps its edge buffers in. */
#define SWEPT_STATIC_SCRATCH_BYTES (8u << 20)

/* Swept solve that allocates nothing, for callers that cannot call cudaMalloc
 * (their device memory belongs to an outside memory manager, or they run in a
 * loop where cudaMalloc/cudaFree would synchronise the device).  The paper has
 * no counterpart; it is swept_step_n with the edge buffers in one fixed 8 MiB
 * device array inside the library instead of a bound workspace, and without a
 * handle, graph or stream of its own.  The array is SWEPT_STATIC_SCRATCH_BYTES
 * (8 MiB) long.
 *   cfg      as for swept_init, except that tile_w must be set (> 0); the
 *            launch options chunk, persistent, cluster and warp_tiles are
 *            ignored (one launch per pass, tiers in shared memory, one point
 *            per thread per trip), which changes no result
 *   u_dev    caller-owned state (layout above), advanced nsteps in place
 * The grid must fit the array: 4 * n * C * sizeof(value) <= SWEPT_STATIC_SCRATCH_BYTES
 * (n <= 2^18 for FP64 heat/KS, 2^19 for FP32); larger grids return
 * SWEPT_ENOMEM_WORKSPACE and launch nothing.  Results equal swept_step_n bit
 * for bit.  Tiles whose shared memory exceeds 48 KB raise the kernels' opt-in
 * limit, never lower it, so handles with larger tiles keep working.
 * The first call on each device looks up the array's device address with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture.  cudaDeviceReset unloads the module, so the
 * kept address is then stale: do not call this entry point again in a process
 * that has reset a device it used.  Every call shares the one array (it keeps
 * the last call's contents), so calls that overlap on the GPU race; serialise
 * them.
 * Errors: SWEPT_EINVAL, SWEPT_ENOMEM_WORKSPACE, SWEPT_ECUDA. */
swept_status swept_step_n_static(const swept_config* cfg, void* u_dev, int64_t nsteps, void* stream);

/* Plan report. */
swept_status swept_get_plan(const swept_handle* h, swept_plan_info* out);

/* Options of the persistent single-problem kernel (persistent = 1); the paper
 * has no counterpart.  Setting one drops the handle's cached graphs.
 *   SWEPT_OPT_SPIN_LIMIT  polls a block makes while waiting for an input tile
 *                         before it gives up and the solve reports
 *                         SWEPT_ETIMEOUT through swept_sync_status (default
 *                         2^24, each poll sleeping about 0.1 us; 1 .. 2^32 - 1)
 *   SWEPT_OPT_START_ITEM  first queue item the kernel claims (default 0).  A
 *                         value > 0 skips the items before it, so later items
 *                         wait for tiles nobody computes: it exists to exercise
 *                         the timeout path without a GPU fault (the state is
 *                         then not a valid solve).
 * Errors: SWEPT_EINVAL (unknown option or value out of range). */
enum { SWEPT_OPT_SPIN_LIMIT = 1, SWEPT_OPT_START_ITEM = 2 };
swept_status swept_set_option(swept_handle* h, int32_t option, int64_t value);

/*
 * Debug build.  libswept_debug.so is the same library compiled with device-side
 * index checks: every window position, tier range, edge / strip / band index,
 * state coordinate, awaited counter and tape slot a kernel computes is checked
 * before use.  A failing check skips the access and records the first failure
 * (no trap).
 *
 * swept_debug_status: *enabled = 1 in the debug build, 0 otherwise.  In the
 * debug build it then synchronizes the device, reads and clears every record:
 * SWEPT_OK if no check failed since the last call, else SWEPT_EDEVICE with the
 * first failure's check id (*check: 1 window, 2 edge, 3 level range, 4 state
 * coordinate, 5 strip, 6 band, 7 counter, 8 tape slot, 9 probe) and index
 * (*index).  SWEPT_ECUDA if the device cannot be read.  Pointers may be NULL.
 *
 * swept_debug_probe: exercises the recording path.  For i < n it copies
 * buf[i] to buf[i] (device array of n doubles) behind a check of i < bound,
 * 0 <= bound <= n, so the checks of i >= bound fail and skip a copy that would
 * have been in range anyway.  Asynchronous on the stream; SWEPT_EINVAL for
 * bad arguments.
 */
swept_status swept_debug_status(int32_t* enabled, int32_t* check, int64_t* index);
swept_status swept_debug_probe(double* buf, int64_t n, int64_t bound, void* stream);

/* Synchronize `stream`, then read and clear the device-side error word.
 * Returns SWEPT_OK, SWEPT_ETIMEOUT or SWEPT_EDEVICE. */
swept_status swept_sync_status(swept_handle* h, void* stream);

/* Host-only check of the swept schedule (no GPU work): replays the index
 * arithmetic the kernels use for nsteps full timesteps on symbolic
 * (point, sub-timestep) tags and verifies that every point of every
 * sub-timestep is computed exactly once, only after all of its stencil inputs,
 * and that the final tier is complete.  With persistent = 1 it replays the
 * persistent kernel's item queue instead and also checks the order its waits
 * guarantee: every read of a state or edge value happens after the item that
 * wrote it, and every write after the previous writer and all items that read
 * the previous value (at most 8192 items; larger returns SWEPT_EINVAL).  Without
 * it, no two blocks of one launch may touch a location one of them writes.
 * computed_out (may be NULL) receives the number of point updates performed.
 * Returns SWEPT_OK or SWEPT_EDEVICE with a message in swept_last_error. */
swept_status swept_check_schedule(swept_handle* h, int64_t nsteps, int64_t* computed_out);

/* Copy the last error message (NUL-terminated, truncated to len). */
swept_status swept_last_error(const swept_handle* h, char* buf, size_t len);

/* Destroy the handle and its cached graphs; NULL is a no-op. */
void swept_free(swept_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SWEPT_H */
