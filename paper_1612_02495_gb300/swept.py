"""Python binding of libswept.so (the C ABI declared in include/swept.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The binding refuses to
load (ImportError) when libswept.so has not been built; there is no fallback.

Functions with the C names take plain integers / pointers, exactly like the
C ABI.  `Solver` is a small convenience owner of a handle plus a torch
workspace tensor.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SWEPT_DEBUG=1 selects the build with device-side index checks (include/swept.h, "Debug build")
DEBUG_BUILD = os.environ.get("SWEPT_DEBUG", "0") == "1"
LIB_PATH = os.path.join(HERE, "libswept_debug.so" if DEBUG_BUILD else "libswept.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("%s is not built (run __graft_entry__.build() or python -m paper_1612_02495_gb300.build%s); "
                      "the CUDA path has no fallback" % (os.path.basename(LIB_PATH), " --debug" if DEBUG_BUILD else ""))

_lib = ctypes.CDLL(LIB_PATH)

# enums (include/swept.h)
SWEPT_OK, SWEPT_EINVAL, SWEPT_ENOMEM_WORKSPACE, SWEPT_ECUDA = 0, 1, 2, 3
SWEPT_ETIMEOUT, SWEPT_EUNSUPPORTED, SWEPT_ENOWORKSPACE, SWEPT_EDEVICE = 4, 5, 6, 7
HEAT, KS, EULER = 0, 1, 2
F32, F64 = 0, 1
BC_PERIODIC, BC_REFLECTIVE = 0, 1

STATUS_NAMES = {0: "SWEPT_OK", 1: "SWEPT_EINVAL", 2: "SWEPT_ENOMEM_WORKSPACE", 3: "SWEPT_ECUDA",
                4: "SWEPT_ETIMEOUT", 5: "SWEPT_EUNSUPPORTED", 6: "SWEPT_ENOWORKSPACE", 7: "SWEPT_EDEVICE"}


class swept_config(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("dtype", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("n", ctypes.c_int64), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("param", ctypes.c_double * 4), ("tile_w", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("chunk", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("warp_tiles", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class swept_plan_info(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("threads", ctypes.c_int32), ("half_cycle", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("stages", ctypes.c_int32), ("components", ctypes.c_int32),
                ("tiles", ctypes.c_int64), ("smem_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("chunk", ctypes.c_int32), ("persistent", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("warp_tiles", ctypes.c_int32), ("last_tile_extra", ctypes.c_int32)]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


swept_init = _sig("swept_init", [ctypes.POINTER(swept_config), ctypes.POINTER(_H)])
swept_workspace_size = _sig("swept_workspace_size", [_H, ctypes.POINTER(_SZ)])
swept_bind_workspace = _sig("swept_bind_workspace", [_H, _P, _SZ])
swept_step_n = _sig("swept_step_n", [_H, _P, _I64, _P])
classic_step_n = _sig("classic_step_n", [_H, _P, _I64, _P])
swept_run_host = _sig("swept_run_host", [_H, _P, _P, _P, _I64, _I32, _P])
swept_adjoint_ckpt_size = _sig("swept_adjoint_ckpt_size", [_H, _I64, ctypes.POINTER(_SZ)])
swept_forward_ckpt = _sig("swept_forward_ckpt", [_H, _P, _I64, _P, _SZ, _P])
swept_adjoint = _sig("swept_adjoint", [_H, _P, _P, _I64, _P, _P, _P, _SZ, _P])
swept_profile_passes = _sig("swept_profile_passes", [_H, _P, _I64, _P, ctypes.POINTER(ctypes.c_double),
                                                     ctypes.POINTER(_I64)])
swept_step_n_static = _sig("swept_step_n_static", [ctypes.POINTER(swept_config), _P, _I64, _P])
swept_get_plan = _sig("swept_get_plan", [_H, ctypes.POINTER(swept_plan_info)])
SWEPT_OPT_SPIN_LIMIT, SWEPT_OPT_START_ITEM = 1, 2
swept_set_option = _sig("swept_set_option", [_H, _I32, _I64])


class swept_batch_problem(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("n", ctypes.c_int64),
                ("nsteps", ctypes.c_int64), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("param", ctypes.c_double)]


SWEPT_BATCH_SPIN_LIMIT, SWEPT_BATCH_START_ITEM, SWEPT_BATCH_GRID = 1, 2, 3
swept_batch_plan = _sig("swept_batch_plan", [ctypes.POINTER(swept_batch_problem), _I64, _I32, _I32,
                                             ctypes.POINTER(_H)])
swept_batch_sizes = _sig("swept_batch_sizes", [_H, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_SZ),
                                               ctypes.POINTER(_I64)])
swept_batch_bind_workspace = _sig("swept_batch_bind_workspace", [_H, _P, _SZ])
swept_batch_set_option = _sig("swept_batch_set_option", [_H, _I32, _I64])
swept_batch_run = _sig("swept_batch_run", [_H, _P, _P])
swept_batch_run_classic = _sig("swept_batch_run_classic", [_H, _P, _P])
swept_batch_sync_status = _sig("swept_batch_sync_status", [_H, _P])
swept_batch_last_error = _sig("swept_batch_last_error", [_H, ctypes.c_char_p, _SZ])
swept_batch_free = _sig("swept_batch_free", [_H], None)
swept_sync_status = _sig("swept_sync_status", [_H, _P])
swept_check_schedule = _sig("swept_check_schedule", [_H, _I64, ctypes.POINTER(_I64)])
swept_last_error = _sig("swept_last_error", [_H, ctypes.c_char_p, _SZ])
swept_free = _sig("swept_free", [_H], None)


class SweptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def last_error(h):
    buf = ctypes.create_string_buffer(512)
    swept_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


def check(status, h=None, what=""):
    if status != SWEPT_OK:
        raise SweptError(status, (what + ": " if what else "") + (last_error(h) if h else ""))


def make_config(scheme, dtype, n, dx, dt, param0, bc=BC_PERIODIC, tile_w=0, threads=0, chunk=0, persistent=0,
                cluster=0, warp_tiles=0):
    c = swept_config()
    c.scheme, c.dtype, c.bc, c.n = int(scheme), int(dtype), int(bc), int(n)
    c.dx, c.dt = float(dx), float(dt)
    c.param[0] = float(param0)
    c.tile_w, c.threads, c.chunk, c.persistent = int(tile_w), int(threads), int(chunk), int(persistent)
    c.cluster = int(cluster)
    c.warp_tiles = int(warp_tiles)
    return c


def init(cfg):
    """swept_init -> handle (int); raises SweptError."""
    h = _H()
    st = swept_init(ctypes.byref(cfg), ctypes.byref(h))
    if st != SWEPT_OK:
        raise SweptError(st, "swept_init rejected the configuration")
    return h.value


def plan(h):
    p = swept_plan_info()
    check(swept_get_plan(h, ctypes.byref(p)), h, "swept_get_plan")
    return {f: getattr(p, f) for f, _ in p._fields_}


def check_schedule(h, nsteps):
    """Host-only symbolic replay of the swept schedule; returns point updates performed."""
    n = _I64()
    check(swept_check_schedule(h, int(nsteps), ctypes.byref(n)), h, "swept_check_schedule")
    return n.value


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """A handle plus its workspace (a torch uint8 tensor on the current device).

    u tensors are contiguous torch tensors on the device with dtype float32 /
    float64 matching `dtype`, shape (n,) for heat/KS and (3, n) for Euler.
    """

    def __init__(self, scheme, dtype, n, dx, dt, param0, bc=BC_PERIODIC, tile_w=0, threads=0, chunk=0, persistent=0,
                 cluster=0, warp_tiles=0):
        import torch

        self.cfg = make_config(scheme, dtype, n, dx, dt, param0, bc, tile_w, threads, chunk, persistent, cluster,
                               warp_tiles)
        self.h = init(self.cfg)
        self.scheme, self.dtype, self.n = scheme, dtype, n
        self.torch_dtype = torch.float32 if dtype == F32 else torch.float64
        sz = _SZ()
        check(swept_workspace_size(self.h, ctypes.byref(sz)), self.h, "swept_workspace_size")
        self.ws = torch.empty(int(sz.value), dtype=torch.uint8, device="cuda")
        check(swept_bind_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr()), sz.value), self.h,
              "swept_bind_workspace")
        self.plan = plan(self.h)

    def _check_u(self, u):
        if not u.is_cuda or not u.is_contiguous() or u.dtype != self.torch_dtype:
            raise ValueError("u must be a contiguous CUDA tensor of dtype %s" % self.torch_dtype)
        want = self.n * (3 if self.scheme == EULER else 1)
        if u.numel() != want:
            raise ValueError("u has %d values, expected %d" % (u.numel(), want))

    def step(self, u, nsteps, stream=None):
        """swept_step_n on u in place (asynchronous on the stream)."""
        self._check_u(u)
        check(swept_step_n(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream_ptr(stream)), self.h,
              "swept_step_n")
        return u

    def classic(self, u, nsteps, stream=None):
        """classic_step_n on u in place (asynchronous on the stream)."""
        self._check_u(u)
        check(classic_step_n(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream_ptr(stream)), self.h,
              "classic_step_n")
        return u

    def run_host(self, u_host_in, u_host_out, u_dev, nsteps, use_swept=True, stream=None):
        """swept_run_host: host tensors in/out (pinned for async copies), u_dev scratch on the device."""
        self._check_u(u_dev)
        check(swept_run_host(self.h, ctypes.c_void_p(u_host_in.data_ptr()), ctypes.c_void_p(u_host_out.data_ptr()),
                             ctypes.c_void_p(u_dev.data_ptr()), int(nsteps), 1 if use_swept else 0,
                             _stream_ptr(stream)), self.h, "swept_run_host")
        return u_host_out

    def profile_passes(self, u, nsteps, stream=None):
        """swept_profile_passes: per-kind (ms, launches) for up, diamond, down, remainder."""
        self._check_u(u)
        ms = (ctypes.c_double * 4)()
        cnt = (_I64 * 4)()
        check(swept_profile_passes(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream_ptr(stream), ms, cnt),
              self.h, "swept_profile_passes")
        names = ("up", "diamond", "down", "remainder")
        return {names[i]: (ms[i], cnt[i]) for i in range(4)}

    def ckpt_size(self, nsteps):
        """swept_adjoint_ckpt_size: checkpoint bytes for the default segment length."""
        sz = _SZ()
        check(swept_adjoint_ckpt_size(self.h, int(nsteps), ctypes.byref(sz)), self.h, "swept_adjoint_ckpt_size")
        return int(sz.value)

    def forward_ckpt(self, u, nsteps, ckpt, stream=None):
        """swept_forward_ckpt: advance u in place and record checkpoints into ckpt (uint8 CUDA tensor)."""
        self._check_u(u)
        check(swept_forward_ckpt(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), ctypes.c_void_p(ckpt.data_ptr()),
                                 ckpt.numel(), _stream_ptr(stream)), self.h, "swept_forward_ckpt")
        return u

    def adjoint(self, gT, nsteps, ckpt, u0=None, g_u0=None, g_param=None, stream=None):
        """swept_adjoint -> (dL/du0 tensor, dL/dparam 1-element float64 tensor)."""
        import torch

        self._check_u(gT)
        g_u0 = torch.empty_like(gT) if g_u0 is None else g_u0
        g_param = torch.zeros(1, dtype=torch.float64, device=gT.device) if g_param is None else g_param
        check(swept_adjoint(self.h, ctypes.c_void_p(u0.data_ptr()) if u0 is not None else None,
                            ctypes.c_void_p(gT.data_ptr()), int(nsteps), ctypes.c_void_p(g_u0.data_ptr()),
                            ctypes.c_void_p(g_param.data_ptr()), ctypes.c_void_p(ckpt.data_ptr()), ckpt.numel(),
                            _stream_ptr(stream)), self.h, "swept_adjoint")
        return g_u0, g_param

    def sync_status(self, stream=None):
        check(swept_sync_status(self.h, _stream_ptr(stream)), self.h, "swept_sync_status")

    def check_schedule(self, nsteps):
        return check_schedule(self.h, nsteps)

    def set_option(self, option, value):
        """swept_set_option (persistent kernel: SWEPT_OPT_SPIN_LIMIT, SWEPT_OPT_START_ITEM)."""
        check(swept_set_option(self.h, int(option), int(value)), self.h, "swept_set_option")

    def close(self):
        if self.h:
            swept_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SweptSolve:
    """Differentiable swept solve: u(T) = solve(u0, param) for nsteps steps.

    `SweptSolve.apply(u0, param, nsteps, scheme=KS, bc=BC_PERIODIC, dx=..., dt=..., tile_w=0, ckpt_bytes=0)`
    returns u(T) (a new tensor).  The backward pass returns dL/du0 and dL/dparam
    through the library's adjoint (swept_adjoint): KS (param = nu) or heat
    (param = alpha), FP64.  The forward pass records checkpoints
    (swept_forward_ckpt); ckpt_bytes = 0 uses swept_adjoint_ckpt_size.
    """

    @staticmethod
    def apply(u0, param, nsteps, **kw):
        return _swept_solve_fn().apply(u0, param, nsteps, kw)


_FN = None


def _swept_solve_fn():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0, param, nsteps, kw):
            scheme = kw.get("scheme", KS)
            sol = Solver(scheme, F64, u0.shape[-1], kw["dx"], kw["dt"], float(param), bc=kw.get("bc", BC_PERIODIC),
                         tile_w=kw.get("tile_w", 0), threads=kw.get("threads", 0))
            nbytes = kw.get("ckpt_bytes", 0) or sol.ckpt_size(nsteps)
            ckpt = torch.empty(int(nbytes), dtype=torch.uint8, device=u0.device)
            u = u0.detach().clone().contiguous()
            sol.forward_ckpt(u, nsteps, ckpt)
            ctx.sol, ctx.ckpt, ctx.nsteps = sol, ckpt, nsteps
            ctx.param_shape = param.shape if torch.is_tensor(param) else None
            ctx.param_device = param.device if torch.is_tensor(param) else None
            return u

        @staticmethod
        def backward(ctx, gT):
            # the handle and its checkpoints stay alive with ctx (a second backward, as with
            # retain_graph=True, continues from the same checkpoints); the Solver frees its
            # handle when ctx is released
            g_u0, g_param = ctx.sol.adjoint(gT.contiguous(), ctx.nsteps, ctx.ckpt)
            gp = g_param.reshape(ctx.param_shape).to(ctx.param_device) if ctx.param_shape is not None else None
            return g_u0, gp, None, None

    _FN = _Fn
    return _FN


def _batch_error(b):
    buf = ctypes.create_string_buffer(512)
    swept_batch_last_error(b, buf, 512)
    return buf.value.decode(errors="replace")


class Batch:
    """A planned batch plus its workspace.

    problems: sequence of dicts with keys scheme (HEAT/KS), n, nsteps, dx, dt,
    param and optionally tile_w.  All states live in one 1-D tensor of
    `state_values` values; problem i occupies [offsets[i], offsets[i] + n_i).
    """

    def __init__(self, problems, dtype, threads=0):
        import torch

        arr = (swept_batch_problem * len(problems))()
        for i, q in enumerate(problems):
            a = arr[i]
            a.scheme, a.tile_w = int(q["scheme"]), int(q.get("tile_w", 0))
            a.n, a.nsteps = int(q["n"]), int(q["nsteps"])
            a.dx, a.dt, a.param = float(q["dx"]), float(q["dt"]), float(q["param"])
        h = _H()
        st = swept_batch_plan(arr, len(problems), int(dtype), int(threads), ctypes.byref(h))
        if st != SWEPT_OK:
            raise SweptError(st, "swept_batch_plan rejected the problems")
        self.b = h.value
        self.count = len(problems)
        self.ns = [int(q["n"]) for q in problems]
        self.dtype = dtype
        self.torch_dtype = torch.float32 if dtype == F32 else torch.float64
        offs = (_I64 * len(problems))()
        sv, wb, items = _I64(), _SZ(), _I64()
        self._check(swept_batch_sizes(self.b, offs, ctypes.byref(sv), ctypes.byref(wb), ctypes.byref(items)))
        self.offsets = [int(x) for x in offs]
        self.state_values, self.items = int(sv.value), int(items.value)
        self.ws = torch.empty(max(int(wb.value), 256), dtype=torch.uint8, device="cuda")
        self._check(swept_batch_bind_workspace(self.b, ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel()))

    def _check(self, st):
        if st != SWEPT_OK:
            raise SweptError(st, _batch_error(self.b))

    def pack(self, states):
        """Host arrays (one per problem) -> device batch state tensor."""
        import numpy as np
        import torch

        host = np.zeros(self.state_values, dtype=np.float64 if self.dtype == F64 else np.float32)
        for o, n, x in zip(self.offsets, self.ns, states):
            host[o:o + n] = x
        return torch.from_numpy(host).cuda()

    def unpack(self, u):
        h = u.cpu().numpy()
        return [h[o:o + n].copy() for o, n in zip(self.offsets, self.ns)]

    def set_option(self, option, value):
        self._check(swept_batch_set_option(self.b, int(option), int(value)))

    def run(self, u, stream=None):
        if not u.is_cuda or u.dtype != self.torch_dtype or u.numel() < self.state_values:
            raise ValueError("batch state must be a CUDA tensor of %d values of %s" % (self.state_values,
                                                                                      self.torch_dtype))
        self._check(swept_batch_run(self.b, ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream)))
        return u

    def run_classic(self, u, stream=None):
        """swept_batch_run_classic: the same advance with the classic decomposition."""
        if not u.is_cuda or u.dtype != self.torch_dtype or u.numel() < self.state_values:
            raise ValueError("batch state must be a CUDA tensor of %d values of %s" % (self.state_values,
                                                                                      self.torch_dtype))
        self._check(swept_batch_run_classic(self.b, ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream)))
        return u

    def sync_status(self, stream=None):
        self._check(swept_batch_sync_status(self.b, _stream_ptr(stream)))

    def close(self):
        if self.b:
            swept_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- 2D (include/swept2d.h)
class swept2d_config(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("bc", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("alpha", ctypes.c_double),
                ("tile_w", ctypes.c_int32), ("threads", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class swept2d_plan_info(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("threads", ctypes.c_int32), ("half_cycle", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("tiles_x", ctypes.c_int64), ("tiles_y", ctypes.c_int64),
                ("smem_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]


swept2d_init = _sig("swept2d_init", [ctypes.POINTER(swept2d_config), ctypes.POINTER(_H)])
swept2d_workspace_size = _sig("swept2d_workspace_size", [_H, ctypes.POINTER(_SZ)])
swept2d_bind_workspace = _sig("swept2d_bind_workspace", [_H, _P, _SZ])
swept2d_step_n = _sig("swept2d_step_n", [_H, _P, _I64, _P])
classic2d_step_n = _sig("classic2d_step_n", [_H, _P, _I64, _P])
swept2d_get_plan = _sig("swept2d_get_plan", [_H, ctypes.POINTER(swept2d_plan_info)])
swept2d_check_schedule = _sig("swept2d_check_schedule", [_H, _I64, ctypes.POINTER(_I64)])
swept2d_last_error = _sig("swept2d_last_error", [_H, ctypes.c_char_p, _SZ])
swept_debug_status = _sig("swept_debug_status", [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(_I64)])
swept_debug_probe = _sig("swept_debug_probe", [_P, _I64, _I64, _P])
DEBUG_CHECK_NAMES = {1: "window", 2: "edge", 3: "level range", 4: "state coordinate", 5: "strip", 6: "band",
                     7: "counter", 8: "tape slot", 9: "probe"}
swept2d_set_option = _sig("swept2d_set_option", [_H, ctypes.c_int32, _I64])
swept2d_sync_status = _sig("swept2d_sync_status", [_H, _P])
SWEPT2D_OPT_CHECK_DROP_WAIT = 16
swept2d_free = _sig("swept2d_free", [_H], None)


def make_config2d(dtype, nx, ny, dx, dt, alpha, tile_w=0, threads=0, bc=BC_PERIODIC, persistent=0):
    c = swept2d_config()
    c.dtype, c.bc, c.nx, c.ny = int(dtype), int(bc), int(nx), int(ny)
    c.dx, c.dt, c.alpha = float(dx), float(dt), float(alpha)
    c.tile_w, c.threads, c.persistent = int(tile_w), int(threads), int(persistent)
    return c


def _err2d(h):
    buf = ctypes.create_string_buffer(512)
    swept2d_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


class Solver2D:
    """A 2D swept handle plus its workspace (a torch uint8 tensor on the current
    device).  States are contiguous CUDA tensors of shape (ny, nx)."""

    def __init__(self, dtype, nx, ny, dx, dt, alpha, tile_w=0, threads=0, bc=BC_PERIODIC, persistent=0):
        import torch

        self.cfg = make_config2d(dtype, nx, ny, dx, dt, alpha, tile_w, threads, bc, persistent)
        h = _H()
        st = swept2d_init(ctypes.byref(self.cfg), ctypes.byref(h))
        if st != SWEPT_OK:
            raise SweptError(st, "swept2d_init rejected the configuration")
        self.h = h.value
        self.nx, self.ny = nx, ny
        self.torch_dtype = torch.float32 if dtype == F32 else torch.float64
        sz = _SZ()
        self._check(swept2d_workspace_size(self.h, ctypes.byref(sz)), "swept2d_workspace_size")
        self.ws = torch.empty(int(sz.value), dtype=torch.uint8, device="cuda")
        self._check(swept2d_bind_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr()), sz.value),
                    "swept2d_bind_workspace")
        p = swept2d_plan_info()
        self._check(swept2d_get_plan(self.h, ctypes.byref(p)), "swept2d_get_plan")
        self.plan = {f: getattr(p, f) for f, _ in p._fields_}

    def _check(self, st, what):
        if st != SWEPT_OK:
            raise SweptError(st, what + ": " + _err2d(self.h))

    def _check_u(self, u):
        if not u.is_cuda or not u.is_contiguous() or u.dtype != self.torch_dtype or u.numel() != self.nx * self.ny:
            raise ValueError("u must be a contiguous CUDA tensor of %d values of dtype %s"
                             % (self.nx * self.ny, self.torch_dtype))

    def step(self, u, nsteps, stream=None):
        """swept2d_step_n on u in place (asynchronous on the stream)."""
        self._check_u(u)
        self._check(swept2d_step_n(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream_ptr(stream)),
                    "swept2d_step_n")
        return u

    def classic(self, u, nsteps, stream=None):
        """classic2d_step_n on u in place (asynchronous on the stream)."""
        self._check_u(u)
        self._check(classic2d_step_n(self.h, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream_ptr(stream)),
                    "classic2d_step_n")
        return u

    def set_option(self, option, value):
        """swept2d_set_option (SWEPT_OPT_SPIN_LIMIT, SWEPT_OPT_START_ITEM)."""
        self._check(swept2d_set_option(self.h, int(option), int(value)), "swept2d_set_option")

    def sync_status(self, stream=None):
        """swept2d_sync_status: raises SweptError(SWEPT_ETIMEOUT) if a persistent wait ran out."""
        self._check(swept2d_sync_status(self.h, _stream_ptr(stream)), "swept2d_sync_status")

    def close(self):
        if self.h:
            swept2d_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_schedule2d(dtype, nx, ny, tile_w, nsteps, threads=0, bc=BC_PERIODIC, persistent=0, drop_wait=-1):
    """Host-only symbolic replay of the 2D launch sequence, or of the persistent
    queue (no GPU): returns the number of point updates, raises SweptError with
    the first violation.  drop_wait >= 0 drops the last wait of that queue item."""
    cfg = make_config2d(dtype, nx, ny, 1.0, 0.2, 1.0, tile_w, threads, bc, persistent)
    h = _H()
    st = swept2d_init(ctypes.byref(cfg), ctypes.byref(h))
    if st != SWEPT_OK:
        raise SweptError(st, "swept2d_init rejected the configuration")
    try:
        if drop_wait >= 0:
            st = swept2d_set_option(h.value, SWEPT2D_OPT_CHECK_DROP_WAIT, int(drop_wait))
            if st != SWEPT_OK:
                raise SweptError(st, _err2d(h.value))
        n = _I64()
        st = swept2d_check_schedule(h.value, int(nsteps), ctypes.byref(n))
        if st != SWEPT_OK:
            raise SweptError(st, _err2d(h.value))
        return n.value
    finally:
        swept2d_free(h.value)


def debug_status():
    """swept_debug_status: (enabled, None) when no check failed since the last
    call, else (enabled, (check name, index)).  Raises SweptError(SWEPT_ECUDA)
    if the device cannot be read."""
    en, chk, idx = ctypes.c_int32(), ctypes.c_int32(), _I64()
    st = swept_debug_status(ctypes.byref(en), ctypes.byref(chk), ctypes.byref(idx))
    if st == SWEPT_OK:
        return bool(en.value), None
    if st == SWEPT_EDEVICE:
        return bool(en.value), (DEBUG_CHECK_NAMES.get(chk.value, str(chk.value)), idx.value)
    raise SweptError(st, "swept_debug_status")


# ---------------------------------------------------------------------------
# one grid split over ranks (include/swept_slab.h): the multi-GPU swept solver
# ---------------------------------------------------------------------------
class swept_slab_layout(ctypes.Structure):
    _fields_ = [("first_block", _I64), ("blocks", _I64), ("x0", _I64), ("x1", _I64), ("state_len", _I64),
                ("edge_values", _I64), ("e0_offset", _I64), ("e1_offset", _I64), ("workspace_bytes", _I64),
                ("tile_w", _I32), ("threads", _I32), ("half_cycle", _I32), ("value_bytes", _I32)]


class swept_slab_xfer(ctypes.Structure):
    _fields_ = [("peer", _I32), ("recv", _I32), ("region", _I32), ("reserved", _I32), ("offset", _I64),
                ("count", _I64)]


swept_slab_init = _sig("swept_slab_init", [ctypes.POINTER(swept_config), _I32, _I32, ctypes.POINTER(_H)])
swept_slab_get_layout = _sig("swept_slab_get_layout", [_H, ctypes.POINTER(swept_slab_layout)])
swept_slab_bind_workspace = _sig("swept_slab_bind_workspace", [_H, _P, _SZ])
swept_slab_launch_count = _sig("swept_slab_launch_count", [_H, _I64, ctypes.POINTER(_I64)])
swept_slab_launch = _sig("swept_slab_launch", [_H, _P, _I64, _I64, _P])
swept_slab_xfers = _sig("swept_slab_xfers", [_H, _I64, _I64, ctypes.POINTER(swept_slab_xfer), _I32,
                                             ctypes.POINTER(_I32)])
swept_slab_last_error = _sig("swept_slab_last_error", [_H, ctypes.c_char_p, _SZ])
swept_slab_free = _sig("swept_slab_free", [_H], None)
swept_slab_check = _sig("swept_slab_check", [ctypes.POINTER(swept_config), _I32, _I64, ctypes.POINTER(_I64),
                                             ctypes.c_char_p, _SZ])
swept_slab_sym_init = _sig("swept_slab_sym_init", [ctypes.POINTER(swept_config), _I32, _I32, _I64,
                                                   ctypes.POINTER(_H)])
swept_slab_sym_buffer = _sig("swept_slab_sym_buffer", [_H, _I32, ctypes.POINTER(ctypes.POINTER(_I64)),
                                                       ctypes.POINTER(_I64)])
swept_slab_sym_launch = _sig("swept_slab_sym_launch", [_H, _I64, ctypes.c_char_p, _SZ])
swept_slab_sym_finish = _sig("swept_slab_sym_finish", [_H, ctypes.POINTER(_I32), ctypes.c_char_p, _SZ])
swept_slab_sym_free = _sig("swept_slab_sym_free", [_H], None)

REGION_E0, REGION_E1, REGION_STATE = 0, 1, 2


def slab_check(scheme, dtype, n, dx, dt, param0, nranks, nsteps, bc=BC_PERIODIC, tile_w=0, threads=0, chunk=0,
               warp_tiles=0):
    """swept_slab_check: host-only symbolic replay of a solve split over nranks ranks; returns the
    point updates performed, raises SweptError with the first violation."""
    cfg = make_config(scheme, dtype, n, dx, dt, param0, bc, tile_w, threads, chunk, 0, 0, warp_tiles)
    done = _I64()
    msg = ctypes.create_string_buffer(512)
    st = swept_slab_check(ctypes.byref(cfg), int(nranks), int(nsteps), ctypes.byref(done), msg, 512)
    if st != SWEPT_OK:
        raise SweptError(st, "swept_slab_check: " + msg.value.decode(errors="replace"))
    return done.value


def _slab_xfer_list(fn, h, nsteps, i):
    buf = (swept_slab_xfer * 8)()
    n = _I32()
    st = fn(h, int(nsteps), int(i), buf, 8, ctypes.byref(n))
    if st != SWEPT_OK:
        raise SweptError(st, "swept_slab_xfers")
    return [(x.peer, x.recv, x.region, x.offset, x.count) for x in buf[:n.value]]


class Slab:
    """Rank `rank` of a grid of n points split over `nranks` ranks, on the current CUDA device.

    The rank's state is a contiguous tensor of C * layout["state_len"] values (C = 3 for
    Euler): global points [x0, x0 + state_len) of each component; the rank owns [x0, x1)
    before and after a solve.  `step` runs the rank's launches and, after each, hands the
    listed transfers to `transport(xfers, views, launch_index)`, where views[region] is the
    flat tensor a transfer's offset and count index (edge buffer 0, 1, the state)."""

    def __init__(self, scheme, dtype, n, dx, dt, param0, rank, nranks, bc=BC_PERIODIC, tile_w=0, threads=0,
                 chunk=0, warp_tiles=0):
        import torch

        self.cfg = make_config(scheme, dtype, n, dx, dt, param0, bc, tile_w, threads, chunk, 0, 0, warp_tiles)
        h = _H()
        st = swept_slab_init(ctypes.byref(self.cfg), int(rank), int(nranks), ctypes.byref(h))
        if st != SWEPT_OK:
            raise SweptError(st, "swept_slab_init rejected the configuration")
        self.h = h.value
        self.rank, self.nranks, self.n, self.scheme = int(rank), int(nranks), int(n), scheme
        self.C = 3 if scheme == EULER else 1
        self.torch_dtype = torch.float32 if dtype == F32 else torch.float64
        lay = swept_slab_layout()
        self._check(swept_slab_get_layout(self.h, ctypes.byref(lay)), "swept_slab_get_layout")
        self.layout = {f: getattr(lay, f) for f, _ in lay._fields_}
        self.ws = torch.empty(int(lay.workspace_bytes), dtype=torch.uint8, device="cuda")
        self._check(swept_slab_bind_workspace(self.h, ctypes.c_void_p(self.ws.data_ptr()), int(lay.workspace_bytes)),
                    "swept_slab_bind_workspace")
        flat = self.ws.view(self.torch_dtype)
        ev = int(lay.edge_values)
        self._edges = [flat[lay.e0_offset:lay.e0_offset + ev], flat[lay.e1_offset:lay.e1_offset + ev]]

    def _check(self, st, what):
        if st != SWEPT_OK:
            buf = ctypes.create_string_buffer(512)
            swept_slab_last_error(self.h, buf, 512)
            raise SweptError(st, what + ": " + buf.value.decode(errors="replace"))

    def local_state(self, u_global):
        """This rank's state array cut from a whole field (C * n values, any device)."""
        import torch

        L = self.layout
        x0, x1, ul = L["x0"], L["x1"], L["state_len"]
        g = u_global.reshape(self.C, self.n)
        u = torch.zeros(self.C, ul, dtype=self.torch_dtype, device="cuda")
        u[:, :x1 - x0] = g[:, x0:x1].to(device="cuda", dtype=self.torch_dtype)
        return u.reshape(-1).contiguous()

    def owned(self, u_local):
        """The rank's points [x0, x1) of its state array, shape (C, x1 - x0)."""
        L = self.layout
        return u_local.reshape(self.C, L["state_len"])[:, :L["x1"] - L["x0"]]

    def launch_count(self, nsteps):
        c = _I64()
        self._check(swept_slab_launch_count(self.h, int(nsteps), ctypes.byref(c)), "swept_slab_launch_count")
        return c.value

    def xfers(self, nsteps, i):
        return _slab_xfer_list(swept_slab_xfers, self.h, nsteps, i)

    def views(self, u_local):
        return [self._edges[0], self._edges[1], u_local]

    def launch(self, u_local, nsteps, i, stream=None):
        if not u_local.is_cuda or not u_local.is_contiguous() or u_local.dtype != self.torch_dtype or \
                u_local.numel() != self.C * self.layout["state_len"]:
            raise ValueError("u_local must be the rank's contiguous state array (C * state_len values)")
        self._check(swept_slab_launch(self.h, ctypes.c_void_p(u_local.data_ptr()), int(nsteps), int(i),
                                      _stream_ptr(stream)), "swept_slab_launch")

    def step(self, u_local, nsteps, transport, stream=None):
        """Advance the rank's state nsteps timesteps, trading with its neighbours through `transport`."""
        for i in range(self.launch_count(nsteps)):
            self.launch(u_local, nsteps, i, stream)
            xs = self.xfers(nsteps, i)
            if xs:
                transport(xs, self.views(u_local), i)
        return u_local

    def close(self):
        if getattr(self, "h", None):
            swept_slab_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlabSym:
    """The symbolic replay of one rank (swept_slab_sym_*): the same launches and transfers as
    `Slab`, over buffers of (point, sub-timestep) tags, two int64 per value.  views() are torch
    int64 CPU tensors of shape (values, 2) sharing the replay's memory, so a transport moves
    rows [offset, offset + count) exactly as it moves values on the GPU."""

    def __init__(self, scheme, dtype, n, dx, dt, param0, rank, nranks, nsteps, bc=BC_PERIODIC, tile_w=0, threads=0,
                 chunk=0, warp_tiles=0):
        import numpy as np
        import torch

        cfg = make_config(scheme, dtype, n, dx, dt, param0, bc, tile_w, threads, chunk, 0, 0, warp_tiles)
        h = _H()
        st = swept_slab_sym_init(ctypes.byref(cfg), int(rank), int(nranks), int(nsteps), ctypes.byref(h))
        if st != SWEPT_OK:
            raise SweptError(st, "swept_slab_sym_init rejected the configuration")
        self.h = h.value
        self._ph = None
        self.nsteps = int(nsteps)
        try:
            # the launch count and transfer lists come from a slab handle of the same configuration
            ph = _H()
            check(swept_slab_init(ctypes.byref(cfg), int(rank), int(nranks), ctypes.byref(ph)), None,
                  "swept_slab_init")
            self._ph = ph.value
            self._views = []
            for region in range(3):
                p = ctypes.POINTER(_I64)()
                nv = _I64()
                check(swept_slab_sym_buffer(self.h, region, ctypes.byref(p), ctypes.byref(nv)), None,
                      "swept_slab_sym_buffer")
                a = np.ctypeslib.as_array(p, shape=(int(nv.value), 2)) if nv.value else np.zeros((0, 2), np.int64)
                self._views.append(torch.from_numpy(a))
        except Exception:
            self.close()
            raise
        self.n = int(n)

    def launch_count(self, nsteps):
        c = _I64()
        check(swept_slab_launch_count(self._ph, int(nsteps), ctypes.byref(c)), None, "swept_slab_launch_count")
        return c.value

    def xfers(self, nsteps, i):
        return _slab_xfer_list(swept_slab_xfers, self._ph, nsteps, i)

    def views(self, u_local=None):
        return self._views

    def launch(self, u_local, nsteps, i, stream=None):
        msg = ctypes.create_string_buffer(512)
        st = swept_slab_sym_launch(self.h, int(i), msg, 512)
        if st != SWEPT_OK:
            raise SweptError(st, "swept_slab_sym_launch: " + msg.value.decode(errors="replace"))

    def step(self, u_local, nsteps, transport, stream=None):
        return Slab.step(self, u_local, nsteps, transport, stream)

    def finish(self, counts):
        """Check the rank's final state; add its per-(sub-timestep, point) update counts into
        `counts` (a contiguous int32 numpy array of (nsteps S + 1) * n entries)."""
        msg = ctypes.create_string_buffer(512)
        st = swept_slab_sym_finish(self.h, counts.ctypes.data_as(ctypes.POINTER(_I32)), msg, 512)
        if st != SWEPT_OK:
            raise SweptError(st, "swept_slab_sym_finish: " + msg.value.decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            swept_slab_sym_free(self.h)
            self.h = None
        if getattr(self, "_ph", None):
            swept_slab_free(self._ph)
            self._ph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pair_keys(xs):
    """(direction of travel, ordinal) of each transfer: a send to side p travels p, a receive
    from side p travels -p; the k-th message of one direction between two neighbours pairs the
    k-th send with the k-th receive."""
    seen = {}
    keys = []
    for peer, recv, region, offset, count in xs:
        travel = -peer if recv else peer
        k = seen.get((travel, recv), 0)
        seen[(travel, recv)] = k + 1
        keys.append((travel, k))
    return keys


def dist_transport(group=None, stage_on_host=False):
    """A transport over torch.distributed point-to-point messages (NCCL between GPUs, gloo on the
    host): every transfer after one launch is posted in one batch_isend_irecv, in the same
    (direction, ordinal) order on both ends of each message, and waited for before the next
    launch.  One rank (world size 1) copies its sends into its own receives.  The slab's rank
    and nranks must be this process's rank and size in `group` (the default group if None).
    With NCCL the messages run in stream order after the launch that produced them, and the
    current stream waits for them before the next launch.  stage_on_host=True moves each message
    through host memory (device to host before a send, host to device after a receive), for a
    host backend such as gloo between processes whose ranks hold device buffers."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)

    def transport(xs, views, i):
        keys = _pair_keys(xs)
        if world == 1:
            return local_copy([(xs, views)], [keys])
        ops = []
        staged = []
        order = sorted(range(len(xs)), key=lambda j: keys[j])
        for j in order:
            peer, recv, region, offset, count = xs[j]
            travel, k = keys[j]
            v = views[region][offset:offset + count]
            if stage_on_host:
                h = v.cpu() if not recv else torch.empty(v.shape, dtype=v.dtype)
                if recv:
                    staged.append((v, h))
                v = h
            tag = (int(i) * 2 + (0 if travel > 0 else 1)) * 16 + k
            dst = (rank + peer) % world
            if group is not None:
                dst = dist.get_global_rank(group, dst)
            ops.append(dist.P2POp(dist.irecv if recv else dist.isend, v, dst, group, tag))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        for v, h in staged:
            v.copy_(h)

    return transport


def local_copy(rank_xfers, rank_keys=None):
    """Carry out the transfers of ranks that live in one process (rank_xfers[r] = (xfers, views)
    of rank r, in ring order): each send is copied into the receive it pairs with."""
    R = len(rank_xfers)
    keys = rank_keys or [_pair_keys(xs) for xs, _ in rank_xfers]
    for r, (xs, views) in enumerate(rank_xfers):
        for j, (peer, recv, region, offset, count) in enumerate(xs):
            if recv:
                continue
            q = (r + peer) % R
            qxs, qviews = rank_xfers[q]
            for jj, (qpeer, qrecv, qregion, qoffset, qcount) in enumerate(qxs):
                if qrecv and qpeer == -peer and keys[q][jj] == keys[r][j]:
                    if qcount != count:
                        raise RuntimeError("paired transfers differ in size")
                    src = views[region][offset:offset + count]
                    dst = qviews[qregion][qoffset:qoffset + qcount]
                    if src.data_ptr() != dst.data_ptr():
                        dst.copy_(src.clone() if q == r else src)
                    break
            else:
                raise RuntimeError("a send of rank %d has no matching receive" % r)


def run_slabs_local(slabs, states, nsteps, stream=None):
    """All ranks of a split grid in one process (one GPU, one stream): launch i on every rank,
    then the transfers after it as device copies.  For testing the partition on one device."""
    n = slabs[0].launch_count(nsteps)
    for i in range(n):
        for s, u in zip(slabs, states):
            s.launch(u, nsteps, i, stream)
        lists = [(s.xfers(nsteps, i), s.views(u)) for s, u in zip(slabs, states)]
        if any(xs for xs, _ in lists):
            local_copy(lists)
    return states
