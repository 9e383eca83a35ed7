"""A grid split over several ranks (include/swept_slab.h), on the host: the
multi-GPU swept solver the paper names as future work (Section
"Conclusion"), in which ranks trade only triangle edges (Section
"First-order", Fig. collection).  Nothing here needs a GPU.

- swept_slab_check replays whole solves over all ranks symbolically: every
  stencil input holds the right (point, sub-timestep), every point-update
  happens exactly once over all ranks, and every rank ends owning the points
  it started with at the last sub-timestep (heat, KS, Euler; both boundary
  conditions; grids of any size; remainders; 1 to nt ranks).
- The Python driver (Slab.step's loop, local_copy, dist_transport) runs the
  same replay one rank at a time: in one process, and as world-size-2 and -3
  gloo process groups whose messages carry the tags.
- A transport that drops or misplaces a transfer is caught.
"""
import os
import random
import socket
from datetime import timedelta

import numpy as np
import pytest

from paper_1612_02495_gb300 import build as libbuild


@pytest.fixture(scope="module")
def S():
    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


def R_of(S, scheme):
    return 1 if scheme == S.HEAT else 2


def stages(S, scheme):
    return 1 if scheme == S.HEAT else 2


def p0(S, scheme):
    return 1.4 if scheme == S.EULER else 1.0


@pytest.mark.parametrize("scheme,bc,W,n,nranks,nsteps", [
    (0, 0, 64, 1024, 1, 101),
    (0, 0, 64, 1024, 2, 101),
    (0, 0, 64, 1024, 3, 64),
    (0, 1, 64, 1024, 4, 33),
    (0, 1, 32, 1009, 5, 77),      # ragged grid, wide last tile on the last rank
    (0, 0, 32, 1009, 31, 40),     # one or two tiles a rank
    (1, 0, 64, 2048, 2, 40),
    (1, 0, 128, 4099, 3, 97),
    (1, 0, 32, 96, 3, 25),        # every rank one tile
    (2, 1, 64, 1024, 2, 33),
    (2, 1, 32, 1009, 4, 21),
    (2, 0, 64, 640, 5, 19),
])
def test_slab_replay(S, scheme, bc, W, n, nranks, nsteps):
    done = S.slab_check(scheme, S.F64, n, 0.1, 1e-3, p0(S, scheme), nranks, nsteps, bc=bc, tile_w=W)
    assert done == n * nsteps * stages(S, scheme)


def test_slab_replay_random_configurations(S):
    rnd = random.Random(20161208)
    for _ in range(400):
        scheme = rnd.choice([S.HEAT, S.KS, S.EULER])
        bc = 0 if scheme == S.KS else rnd.choice([0, 1])
        R = R_of(S, scheme)
        W = 4 * R * rnd.choice([1, 2, 4, 8])
        nt = rnd.randint(2, 9)
        n = nt * W + rnd.choice([0, 0, 1, W - 1, rnd.randint(0, W - 1)])
        nranks = rnd.randint(1, nt)
        nsteps = rnd.choice([0, 1, 2, rnd.randint(1, 60)])
        done = S.slab_check(scheme, S.F64, n, 0.1, 1e-3, p0(S, scheme), nranks, nsteps, bc=bc, tile_w=W)
        assert done == n * nsteps * stages(S, scheme), (scheme, bc, W, n, nranks, nsteps)


def test_slab_layout_partitions_the_grid(S):
    for scheme, n, W, nranks in [(S.HEAT, 1024, 64, 3), (S.KS, 4099, 128, 5), (S.EULER, 1009, 32, 7)]:
        C = 3 if scheme == S.EULER else 1
        R = R_of(S, scheme)
        h = W // (2 * R)
        E = 2 * h * C * 2 * R
        nt = n // W
        X = n - nt * W
        x_prev, blocks = 0, 0
        for r in range(nranks):
            cfg = S.make_config(scheme, S.F64, n, 0.1, 1e-3, p0(S, scheme), tile_w=W)
            hh = S._H()
            assert S.swept_slab_init(S.ctypes.byref(cfg), r, nranks, S.ctypes.byref(hh)) == S.SWEPT_OK
            lay = S.swept_slab_layout()
            assert S.swept_slab_get_layout(hh.value, S.ctypes.byref(lay)) == S.SWEPT_OK
            S.swept_slab_free(hh.value)
            assert lay.x0 == x_prev and lay.first_block == blocks and lay.blocks >= 1
            assert lay.x1 == (n if r == nranks - 1 else (lay.first_block + lay.blocks) * W)
            assert lay.state_len == lay.x1 - lay.x0 + W // 2
            assert lay.edge_values == min(lay.blocks + 2, nt) * E + (C * X if X else 0)
            assert lay.e1_offset * lay.value_bytes >= lay.edge_values * lay.value_bytes
            assert lay.workspace_bytes >= 2 * lay.edge_values * lay.value_bytes
            x_prev, blocks = lay.x1, blocks + lay.blocks
        assert x_prev == n and blocks == nt


@pytest.mark.parametrize("bad", [
    dict(nranks=0), dict(rank=-1), dict(rank=3, nranks=3), dict(nranks=17),  # 16 tiles
    dict(persistent=1), dict(cluster=1), dict(n=7),  # n = 7: no tiling of two 4-point tiles
])
def test_slab_init_rejects(S, bad):
    kw = dict(rank=0, nranks=2, persistent=0, cluster=0, n=1024)
    kw.update(bad)
    cfg = S.make_config(S.HEAT, S.F64, kw["n"], 0.1, 1e-3, 1.0, tile_w=64 if kw["n"] >= 128 else 0,
                        persistent=kw["persistent"], cluster=kw["cluster"])
    h = S._H()
    st = S.swept_slab_init(S.ctypes.byref(cfg), kw["rank"], kw["nranks"], S.ctypes.byref(h))
    assert st in (S.SWEPT_EINVAL, S.SWEPT_EUNSUPPORTED)
    assert not h.value


def test_slab_xfer_sizes(S):
    """Half an edge block before each diamond-kind pass; W/2 (odd down pass) or
    R rem (gap pass) state values per component after them; nothing else."""
    n, W = 1024, 64
    for scheme in (S.HEAT, S.KS, S.EULER):
        C = 3 if scheme == S.EULER else 1
        R = R_of(S, scheme)
        h = W // (2 * R)
        cfg = S.make_config(scheme, S.F64, n, 0.1, 1e-3, p0(S, scheme), bc=1 if scheme == S.EULER else 0, tile_w=W)
        hh = S._H()
        assert S.swept_slab_init(S.ctypes.byref(cfg), 1, 3, S.ctypes.byref(hh)) == S.SWEPT_OK
        nsteps = (3 * h + 5) // stages(S, scheme) if scheme == S.HEAT else (3 * h + 6) // 2
        n_sub = nsteps * stages(S, scheme)
        q, rem = divmod(n_sub, h)
        cnt = S._I64()
        assert S.swept_slab_launch_count(hh.value, nsteps, S.ctypes.byref(cnt)) == S.SWEPT_OK
        assert cnt.value == (q + 1 if q else 0) + (2 if rem else 0)
        for i in range(cnt.value):
            xs = S._slab_xfer_list(S.swept_slab_xfers, hh.value, nsteps, i)
            edge = [x for x in xs if x[2] != S.REGION_STATE]
            state = [x for x in xs if x[2] == S.REGION_STATE]
            nxt_is_pass = (1 <= i + 1 <= q) or (rem and i + 1 == (q + 1 if q else 0) + 1)
            assert len(edge) == (2 if nxt_is_pass else 0)
            assert all(x[4] == h * C * 2 * R for x in edge)
            if i == q and q % 2 == 1 and q > 0:
                assert len(state) == 2 * C and all(x[4] == W // 2 for x in state)
            elif rem and i == cnt.value - 1:
                assert len(state) == 2 * C and all(x[4] == R * rem for x in state)
            else:
                assert state == []
        S.swept_slab_free(hh.value)


def run_sym_in_process(S, scheme, bc, n, W, nranks, nsteps, transport_filter=None):
    syms = [S.SlabSym(scheme, S.F64, n, 0.1, 1e-3, p0(S, scheme), r, nranks, nsteps, bc=bc, tile_w=W)
            for r in range(nranks)]
    L = syms[0].launch_count(nsteps)
    for i in range(L):
        for s in syms:
            s.launch(None, nsteps, i)
        lists = [(s.xfers(nsteps, i), s.views()) for s in syms]
        if transport_filter:
            lists = transport_filter(i, lists)
        if any(xs for xs, _ in lists):
            S.local_copy(lists)
    counts = np.zeros((nsteps * stages(S, scheme) + 1) * n, dtype=np.int32)
    for s in syms:
        s.finish(counts)
        s.close()
    return counts.reshape(-1, n)


@pytest.mark.parametrize("scheme,bc,n,W,nranks,nsteps", [
    (0, 1, 1009, 32, 3, 71), (1, 0, 1024, 64, 4, 37), (2, 1, 640, 64, 2, 29), (0, 0, 256, 64, 1, 50)])
def test_python_driver_in_process(S, scheme, bc, n, W, nranks, nsteps):
    counts = run_sym_in_process(S, scheme, bc, n, W, nranks, nsteps)
    assert (counts[1:] == 1).all()


def test_dropped_or_misplaced_transfers_are_caught(S):
    def drop_state(i, lists):
        return [([x for x in xs if x[2] != S.REGION_STATE], v) for xs, v in lists]

    def drop_edges(i, lists):
        return [([x for x in xs if x[2] == S.REGION_STATE], v) for xs, v in lists]

    def shift_receive(i, lists):
        out = []
        for xs, v in lists:
            out.append(([(p, rc, rg, off + (1 if rc and rg != S.REGION_STATE else 0), c) for p, rc, rg, off, c in xs], v))
        return out

    for f in (drop_state, drop_edges, shift_receive):
        with pytest.raises(S.SweptError):
            run_sym_in_process(S, S.HEAT, 0, 1024, 64, 3, 101, f)  # q = 3 (odd down pass) + remainder


# --- multi-process: world-size 2 and 3 gloo groups, one rank per process ------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_rank(rank, world, port, case, q, stage=False):
    try:
        import torch
        import torch.distributed as dist

        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
        from paper_1612_02495_gb300 import swept as S

        scheme, bc, n, W, nsteps = case
        sym = S.SlabSym(scheme, S.F64, n, 0.1, 1e-3, 1.4 if scheme == S.EULER else 1.0, rank, world, nsteps, bc=bc,
                        tile_w=W)
        sym.step(None, nsteps, S.dist_transport(stage_on_host=stage))
        counts = np.zeros((nsteps * (1 if scheme == S.HEAT else 2) + 1) * n, dtype=np.int32)
        sym.finish(counts)
        t = torch.from_numpy(counts)
        dist.all_reduce(t)
        sym.close()
        dist.destroy_process_group()
        q.put((rank, "ok", t.numpy().reshape(-1, n)[1:].min(), t.numpy().reshape(-1, n)[1:].max()))
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e), None))


@pytest.mark.parametrize("world,case,stage", [
    (2, (0, 0, 1024, 64, 101), False),   # heat, periodic: odd down pass + remainder
    (2, (1, 0, 2048, 128, 70), False),   # KS
    (3, (0, 1, 1009, 32, 77), False),    # heat, insulated, ragged grid
    (3, (2, 1, 1024, 64, 40), False),    # Euler, reflective walls
    (3, (1, 0, 1536, 128, 55), True),    # messages staged through host buffers
])
def test_gloo_ranks_carry_the_exchange(S, world, case, stage):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_gloo_rank, args=(r, world, port, case, q, stage)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=240) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    for rank, status, a, b in res:
        assert status == "ok", (rank, a)
        assert a == 1 and b == 1, (rank, a, b)


def test_slab_calls_validate_before_touching_a_device(S):
    """Error paths of the slab calls, on the host: no workspace, a launch index out of range,
    a transfer list longer than the caller's array, NULL pointers; without a device a valid
    launch fails with SWEPT_ECUDA instead of launching."""
    import ctypes

    cfg = S.make_config(S.EULER, S.F64, 1024, 1.0 / 1024, 1e-4, 1.4, bc=S.BC_REFLECTIVE, tile_w=64)
    h = S._H()
    assert S.swept_slab_init(ctypes.byref(cfg), 1, 3, ctypes.byref(h)) == S.SWEPT_OK
    h = h.value
    fake = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced on these paths
    assert S.swept_slab_launch(h, fake, 10, 0, None) == S.SWEPT_ENOWORKSPACE
    assert S.swept_slab_launch(h, None, 10, 0, None) == S.SWEPT_EINVAL
    assert S.swept_slab_bind_workspace(h, ctypes.c_void_p(1 << 20 | 8), 1 << 30) == S.SWEPT_EINVAL  # misaligned
    lay = S.swept_slab_layout()
    assert S.swept_slab_get_layout(h, ctypes.byref(lay)) == S.SWEPT_OK
    assert S.swept_slab_bind_workspace(h, fake, lay.workspace_bytes - 1) == S.SWEPT_ENOMEM_WORKSPACE
    assert S.swept_slab_bind_workspace(h, fake, lay.workspace_bytes) == S.SWEPT_OK
    cnt = S._I64()
    assert S.swept_slab_launch_count(h, 10, ctypes.byref(cnt)) == S.SWEPT_OK and cnt.value > 0
    assert S.swept_slab_launch(h, fake, 10, cnt.value, None) == S.SWEPT_EINVAL
    assert S.swept_slab_launch(h, fake, 10, -1, None) == S.SWEPT_EINVAL
    assert S.swept_slab_launch(h, fake, -1, 0, None) == S.SWEPT_EINVAL
    buf = (S.swept_slab_xfer * 8)()
    n = S._I32()
    # 10 Euler steps with h = 16: 20 sub-steps, one odd down pass and a remainder of 4; after the down
    # pass and after the gap pass each of the 3 components is sent and received
    worst = max(range(cnt.value), key=lambda i: len(S._slab_xfer_list(S.swept_slab_xfers, h, 10, i)))
    m = len(S._slab_xfer_list(S.swept_slab_xfers, h, 10, worst))
    assert m >= 2
    assert S.swept_slab_xfers(h, 10, worst, buf, m - 1, ctypes.byref(n)) == S.SWEPT_EINVAL
    assert S.swept_slab_xfers(h, 10, worst, None, 8, ctypes.byref(n)) == S.SWEPT_EINVAL
    assert S.swept_slab_xfers(h, 10, cnt.value + 5, buf, 8, ctypes.byref(n)) == S.SWEPT_OK and n.value == 0
    if not __import__("torch").cuda.is_available():
        assert S.swept_slab_launch(h, fake, 10, 0, None) == S.SWEPT_ECUDA
    S.swept_slab_free(h)
    S.swept_slab_free(None)


def test_slab_check_refuses_oversized_replays(S):
    with pytest.raises(S.SweptError) as e:
        S.slab_check(S.HEAT, S.F64, 1 << 20, 0.1, 1e-3, 1.0, 64, 100, tile_w=1024)  # 101 x 2^20 x 64 > 2e9
    assert e.value.status == S.SWEPT_EINVAL
