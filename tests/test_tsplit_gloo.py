"""The time-slab domain decomposition (paper_1702_00124_gb300.tsplit) with two
gloo ranks on the CPU: each rank holds half the time slices of a 4^3 x 8
lattice, exchanges the two 12-real half-spinor faces the plan prescribes, and
applies the Wilson hop (Section 3.1) to its slab; the assembled result must
equal the oracle's whole-lattice hop, for D and D^dag, and the FP64 all-reduce
of the ranks' partial inner products must equal the whole-lattice one.  The
per-slab arithmetic below is test code (numpy, the oracle's conventions); the
plan, the exchange and the global sum are the module's."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

DIMS = (4, 4, 4, 8)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _upper(v):
    """The two upper spin components (the half spinor) of [..., 4, 3]."""
    return v[..., :2, :]


def _rank(rank, world, port, dagger, out):
    import torch
    import torch.distributed as dist
    from oracle import lattice
    from oracle.dirac import GAMMA
    from oracle.lattice import shift
    from paper_1702_00124_gb300 import synthetic, tsplit
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lx, ly, lz, lt = DIMS
    p = 0                                            # output parity
    U = synthetic.gauge_field(DIMS, 0.5, 881)
    psi = lattice.mask(synthetic.spinor_field(DIMS, 882), DIMS, 1 - p)
    t0, nt = tsplit.slab(lt, rank, world)
    Ul, pl = U[t0:t0 + nt], psi[t0:t0 + nt]
    par = lattice.parity(DIMS)[t0:t0 + nt]
    sg = 1 if dagger else -1                         # forward projector 1 + sg g
    g = GAMMA[3]
    one = np.eye(4)
    Pf, Pb = one + sg * g, one - sg * g

    def spin(m, v):
        return np.einsum("st,...tc->...sc", m, v)

    def colour(Um, v):
        return np.einsum("...ab,...sb->...sa", Um, v)

    def colour_dag(Um, v):
        return np.einsum("...ba,...sb->...sa", Um.conj(), v)

    # faces of the input parity, packed as 12 reals per face site
    m_first = par[0] == 1 - p
    m_last = par[nt - 1] == 1 - p
    face_fwd = _upper(spin(Pf, pl[0]))[m_first]                          # for rank - 1
    face_bwd = _upper(colour_dag(Ul[nt - 1, ..., 3, :, :], spin(Pb, pl[nt - 1])))[m_last]   # for rank + 1
    n = tsplit.face_sites(DIMS)
    assert face_fwd.shape == (n, 2, 3) and face_bwd.shape == (n, 2, 3)
    assert 2 * face_fwd.size * 2 * 8 == tsplit.face_bytes(DIMS, 8)       # complex -> 2 reals, FP64
    tens = [torch.from_numpy(np.ascontiguousarray(f).view(np.float64).copy()) for f in (face_fwd, face_bwd)]
    from_next, from_prev = torch.empty_like(tens[0]), torch.empty_like(tens[1])
    tsplit.exchange_faces(dist, rank, world, tens[0], tens[1], from_next, from_prev)
    h_next = from_next.numpy().view(np.complex128).reshape(n, 2, 3)
    w_prev = from_prev.numpy().view(np.complex128).reshape(n, 2, 3)
    if tsplit.crosses_boundary(rank, world, forward=True):
        h_next = -h_next
    if tsplit.crosses_boundary(rank, world, forward=False):
        w_prev = -w_prev
    o = np.zeros_like(pl)
    for mu in range(3):                              # x, y, z: inside the slab
        gm = GAMMA[mu]
        fw = colour(Ul[..., mu, :, :], shift(pl, mu, +1))
        o += fw + sg * spin(gm, fw)
        bw = colour_dag(shift(Ul[..., mu, :, :], mu, -1), shift(pl, mu, -1))
        o += bw - sg * spin(gm, bw)
    for t in range(nt):                              # t inside the slab
        if t + 1 < nt:
            o[t] += spin(Pf, colour(Ul[t, ..., 3, :, :], pl[t + 1]))
        if t > 0:
            o[t] += spin(Pb, colour_dag(Ul[t - 1, ..., 3, :, :], pl[t - 1]))
    # faces: forward hop of the last slice, backward hop of the first slice
    m_out_last = par[nt - 1] == p
    m_out_first = par[0] == p
    hf = np.zeros((lz, ly, lx, 2, 3), dtype=np.complex128)
    # site (z, y, x) of parity p on the last slice takes the face entry of its
    # forward neighbour, the site (z, y, x) of parity 1-p on the next rank's first slice
    hf[m_first] = h_next
    # in the chiral basis g_t swaps the upper and lower spin pairs, so the lower
    # spins of (1 + s g_t) v are s times its upper spins
    uh = colour(Ul[nt - 1, ..., 3, :, :], hf)
    contrib = np.concatenate([uh, sg * uh], axis=-2)
    o[nt - 1][m_out_last] += contrib[m_out_last]
    wb = np.zeros((lz, ly, lx, 2, 3), dtype=np.complex128)
    wb[m_last] = w_prev
    contrib = np.concatenate([wb, -sg * wb], axis=-2)
    o[0][m_out_first] += contrib[m_out_first]
    o = lattice.mask(np.concatenate([np.zeros((t0,) + o.shape[1:]), o,
                                     np.zeros((lt - t0 - nt,) + o.shape[1:])]), DIMS, p)[t0:t0 + nt]
    dot = tsplit.global_sum(dist, np.vdot(o, o).real)           # |D psi|^2, a CG norm
    out.put((rank, o, dot))
    dist.destroy_process_group()


@pytest.mark.parametrize("dagger", [False, True], ids=["D", "Ddag"])
def test_tsplit_hop_and_global_dot_gloo(dagger):
    from oracle import lattice, wilson
    from paper_1702_00124_gb300 import synthetic
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, dagger, q)) for r in range(2)]
    for pr in ps:
        pr.start()
    res = sorted((q.get(timeout=180) for _ in ps), key=lambda r: r[0])
    for pr in ps:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    U = synthetic.gauge_field(DIMS, 0.5, 881)
    psi = lattice.mask(synthetic.spinor_field(DIMS, 882), DIMS, 1)
    ref = lattice.mask(wilson.hop(U, psi, dagger=dagger), DIMS, 0)
    got = np.concatenate([r[1] for r in res])
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    want = float(np.vdot(ref, ref).real)
    for r in res:
        assert abs(r[2] - want) < 1e-12 * abs(want)


def test_tsplit_plan():
    from paper_1702_00124_gb300 import tsplit
    assert tsplit.slab(64, 3, 4) == (48, 16)
    assert tsplit.neighbours(0, 4) == (1, 3)
    assert tsplit.face_sites((32, 32, 32, 64)) == 16384
    assert tsplit.face_bytes((32, 32, 32, 64), 4) == 2 * 16384 * 12 * 4
    assert tsplit.crosses_boundary(3, 4, True) and tsplit.crosses_boundary(0, 4, False)
    assert not tsplit.crosses_boundary(1, 4, True)
    with pytest.raises(ValueError):
        tsplit.slab(64, 0, 3)
    with pytest.raises(ValueError):
        tsplit.slab(12, 0, 4)                      # slabs of 3 slices: odd
