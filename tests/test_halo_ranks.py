"""The t-slab domain decomposition across processes, on CPU: gloo ranks exchange
spin-projected faces (paper_1109_2935_gb300/halo.py) and each computes the oracle's
Wilson-clover operator on its slab plus ghosts, which must equal the whole-lattice
oracle there; the allreduce of local norms gives the global norm; a rank that never
sends makes the other's exchange end with ERR_TIMEOUT instead of hanging. With four
ranks the previous and the next neighbour of a rank are different processes, so a face
sent the wrong way round would fail the comparison (with two they coincide)."""
import pytest
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

DIMS, KAPPA = (4, 4, 4, 8), 0.13


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _project(psi_slice, s):
    """h = psi_up + s psi_low (the t-projection, B_t = 1): (Z, Y, X, 2, 3)."""
    return psi_slice[..., :2, :] + s * psi_slice[..., 2:, :]


def _worker(rank, world, port, q, done):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import wilson
    from paper_1109_2935_gb300 import synth
    from paper_1109_2935_gb300.halo import HaloExchange, HaloTimeout
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = synth.wilson_gauge(DIMS, 0.5, 1, 4001).numpy()
    psi = synth.wilson_spinor(DIMS, 4002).numpy()
    A = wilson.clover(U, 1.0)
    ref = wilson.apply_M(U, A, KAPPA, psi)            # whole lattice, antiperiodic t
    LT = DIMS[3] // world
    t0 = rank * LT
    loc = psi[t0:t0 + LT]
    hx = HaloExchange(timeout_s=2.0)
    # gauge ghosts once: the previous rank's last-slice t-links
    _, links_prev = hx.exchange(torch.from_numpy(U[t0, ..., 3, :, :].copy()),
                                torch.from_numpy(U[t0 + LT - 1, ..., 3, :, :].copy()))
    # spinor faces: first slice for the previous rank's forward hop (1 - gamma_t),
    # last slice for the next rank's backward hop (1 + gamma_t)
    from_next, from_prev = hx.exchange(torch.from_numpy(_project(loc[0], -1.0)),
                                       torch.from_numpy(_project(loc[-1], +1.0)))
    h_next, h_prev = from_next.numpy().copy(), from_prev.numpy().copy()
    if rank == world - 1:
        h_next *= -1.0                                 # the hop crosses the antiperiodic edge
    if rank == 0:
        h_prev *= -1.0
    # slab plus one ghost slice on each side; a ghost spinor [h; 0] projects to h
    ext = np.zeros((LT + 2,) + loc.shape[1:], dtype=complex)
    ext[1:-1] = loc
    ext[0, ..., :2, :] = h_prev
    ext[-1, ..., :2, :] = h_next
    Uext = np.zeros((LT + 2,) + U.shape[1:], dtype=complex)
    Uext[:] = np.eye(3)
    Uext[1:-1] = U[t0:t0 + LT]
    Uext[0, ..., 3, :, :] = links_prev.numpy()
    Aext = np.zeros((LT + 2,) + A.shape[1:], dtype=complex)
    Aext[1:-1] = A[t0:t0 + LT]
    out = wilson.apply_M(Uext, Aext, KAPPA, ext, antiperiodic_t=False)[1:-1]
    err = float(np.max(np.abs(out - ref[t0:t0 + LT])))
    n2 = hx.allreduce(torch.tensor([float(np.vdot(out, out).real)], dtype=torch.float64)).item()
    n2_ref = float(np.vdot(ref, ref).real)
    dist.barrier()
    # fault, last: rank 1 never joins the next exchange; rank 0's exchange must end with
    # ERR_TIMEOUT. The connection is closed after that, so the ranks part via the host.
    timed_out, code = False, None
    if rank == 0:
        f = torch.zeros(4, dtype=torch.float64)
        try:
            HaloExchange(timeout_s=0.5).exchange(f, f)
        except HaloTimeout as e:
            timed_out, code = True, e.code
        done.set()
    else:
        done.wait(60)
    q.put((rank, err, n2, n2_ref, timed_out, code))


@pytest.mark.parametrize("world", [2, 4])
def test_rank_halo_exchange_matches_whole_lattice_and_times_out(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    done = ctx.Event()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, done)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, err, n2, n2_ref, timed_out, code in got:
        assert err < 1e-13, (rank, err)
        assert abs(n2 - n2_ref) < 1e-12 * n2_ref
    assert got[0][4] and got[0][5] == -8
    assert not any(g[4] for g in got[1:])


def _grid_worker(rank, world, port, grid, q):
    """Rank `rank` of a (g_x, g_y, g_z, g_t) grid: faces and gauge ghosts exchanged in every
    cut dimension, the oracle operator on the block plus one ghost layer per cut side."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import wilson
    from oracle.gamma import GAMMA
    from paper_1109_2935_gb300 import synth
    from paper_1109_2935_gb300.halo import HaloExchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = synth.wilson_gauge(DIMS, 0.5, 1, 4001).numpy()
    psi = synth.wilson_spinor(DIMS, 4002).numpy()
    A = wilson.clover(U, 1.0)
    ref = wilson.apply_M(U, A, KAPPA, psi)            # whole lattice, antiperiodic t
    hx = HaloExchange(timeout_s=5.0, grid=grid)
    co = hx.coords
    ax = lambda mu: 3 - mu                             # arrays are [t, z, y, x, ...]
    loc_len = [DIMS[mu] // grid[mu] for mu in range(4)]
    blk = [slice(None)] * 4
    for mu in range(4):
        blk[ax(mu)] = slice(co[mu] * loc_len[mu], (co[mu] + 1) * loc_len[mu])
    blk = tuple(blk)
    loc, Uloc, Aloc = psi[blk], U[blk], A[blk]
    cut = [mu for mu in range(4) if grid[mu] > 1]
    ext_shape = [loc.shape[a] + (2 if (3 - a) in cut else 0) for a in range(4)]
    inner = tuple(slice(1, -1) if (3 - a) in cut else slice(None) for a in range(4))
    ext = np.zeros(tuple(ext_shape) + loc.shape[4:], dtype=complex)
    Uext = np.zeros(tuple(ext_shape) + U.shape[4:], dtype=complex)
    Uext[:] = np.eye(3)
    Aext = np.zeros(tuple(ext_shape) + A.shape[4:], dtype=complex)
    ext[inner], Uext[inner], Aext[inner] = loc, Uloc, Aloc

    def project(sl, mu, s):   # the two upper spin components of (1 + s gamma_mu) psi
        P = (np.eye(4) + s * GAMMA[mu])[:2]
        return np.einsum("ab,...bc->...ac", P, sl)

    for mu in cut:
        a = ax(mu)
        first, last = np.take(loc, 0, axis=a), np.take(loc, loc_len[mu] - 1, axis=a)
        from_next, from_prev = hx.exchange(torch.from_numpy(project(first, mu, -1.0)),
                                           torch.from_numpy(project(last, mu, +1.0)), mu=mu)
        h_next, h_prev = from_next.numpy().copy(), from_prev.numpy().copy()
        if mu == 3 and co[3] == grid[3] - 1:
            h_next *= -1.0                             # the hop crosses the antiperiodic edge
        if mu == 3 and co[3] == 0:
            h_prev *= -1.0
        ulast = np.take(Uloc, loc_len[mu] - 1, axis=a)[..., mu, :, :].copy()
        _, links_prev = hx.exchange(torch.zeros(1, dtype=torch.complex128), torch.from_numpy(ulast), mu=mu)
        for at, h in ((0, h_prev), (-1, h_next)):
            idx = list(inner)
            idx[a] = at
            ext[tuple(idx) + (slice(0, 2),)] = h       # ghost spinor [h; 0]
        idx = list(inner)
        idx[a] = 0
        Uext[tuple(idx) + (mu,)] = links_prev.numpy()
    out = wilson.apply_M(Uext, Aext, KAPPA, ext, antiperiodic_t=3 not in cut)[inner]
    err = float(np.max(np.abs(out - ref[blk])))
    n2 = hx.allreduce(torch.tensor([float(np.vdot(out, out).real)], dtype=torch.float64)).item()
    dist.barrier()
    q.put((rank, err, n2, float(np.vdot(ref, ref).real)))


@pytest.mark.parametrize("grid", [(1, 1, 2, 2), (2, 2, 1, 1), (2, 1, 1, 2)])
def test_rank_grid_halo_exchange_matches_whole_lattice(grid):
    """Four gloo ranks cutting two dimensions: faces projected for every cut direction and
    the backward gauge ghosts travel to the right neighbours, the antiperiodic sign goes to
    the ranks on the t edge, and every block equals the whole-lattice oracle."""
    world = int(np.prod(grid))
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_grid_worker, args=(r, world, port, grid, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, err, n2, n2_ref in got:
        assert err < 1e-13, (rank, err)
        assert abs(n2 - n2_ref) < 1e-12 * n2_ref


def _grid_check_worker(port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1109_2935_gb300.halo import HaloExchange
    dist.init_process_group("gloo", rank=0, world_size=1)
    out = []
    for grid in ((1, 1, 1, 1), (2, 1, 1, 1), (1, 1, 0, 1), (1, 1, 1)):
        try:
            hx = HaloExchange(grid=grid)
            f = torch.arange(4, dtype=torch.float64)
            a, b = hx.exchange(f, f + 1, mu=2)   # one rank in z: its own faces, no messages
            out.append(("ok", hx.coords, bool(torch.equal(a, f) and torch.equal(b, f + 1))))
        except ValueError:
            out.append(("ValueError",))
    dist.destroy_process_group()
    q.put(out)


def test_rank_grid_must_match_the_world():
    """A grid whose ranks do not multiply to the world size (or has a zero / missing
    dimension) is rejected; in a dimension with one rank the faces are the rank's own."""
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_grid_check_worker, args=(port, q))
    p.start()
    p.join(120)
    assert p.exitcode == 0
    out = q.get(timeout=10)
    assert out[0] == ("ok", (0, 0, 0, 0), True)
    assert out[1:] == [("ValueError",)] * 3
