"""Batched multi-lattice, multi-RHS K_hat and CG against the oracle.

Small batch (three uneven lattices, 1-3 right-hand sides, different kappa):
batched K_hat (FP32, interleaved right-hand sides, one launch for all
lattices) per system vs the oracle (2e-5 per site); batched mixed-precision
CG, with and without CUDA-graph replay and with the reliable updates' K_hat x
in FP64 or double-float, reaches the FP64 true residual 1e-10 recomputed by
the oracle and matches the single-system solve (1e-8).  A second
small batch with four right-hand sides per lattice runs the batched K_hat in
every tile shape (64-256 items per block, one, two or four right-hand sides per
thread of the hop, or the per-thread link-staging pipeline; 2e-5 per site) and
CG with two and four per thread and with link staging, as graph-replayed
launches and as the persistent cooperative kernel (1e-10).

The batched workload at full size (24 lattices: 8 x 8^4, 8 x 12^3 x 24,
8 x 16^3 x 32, links exp(0.4 i H), kappa ~ U[0.125, 0.135], 4 Gaussian
right-hand sides each): every one of the 96 systems reaches 1e-10, checked
with each lattice's FP64 K_hat, with graph-replayed launches and with the
persistent cooperative kernel; the batched K_hat matches the oracle's
sampled-site K_hat on one lattice of each size.
"""
import numpy as np
import pytest

from oracle import lattice, sampled, wilson
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _make(dims, a, kappa, nr, seed, wd, gu, stream, recon=0):
    U = synthetic.gauge_field(dims, a, seed)
    lat = wd.Lattice(dims, stream=stream)
    lat.wd_set_recon(recon)
    lat.wd_gauge_load(gu.dev(U))
    rhs = [lattice.mask(synthetic.spinor_field(dims, seed + 1 + r), dims, 0) for r in range(nr)]
    return U, lat, rhs


@pytest.fixture(scope="module")
def small():
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    spec = [((4, 4, 4, 4), 0.5, 0.12, 2), ((6, 4, 6, 10), 0.4, 0.128, 3), ((8, 8, 8, 8), 0.4, 0.125, 1)]
    stream = torch.cuda.current_stream()
    items = [_make(d, a, k, nr, 900 + 10 * i, wd, gu, stream) for i, (d, a, k, nr) in enumerate(spec)]
    lats = [it[1] for it in items]
    batch = wd.Batch(lats, [s[2] for s in spec], [s[3] for s in spec])
    yield spec, items, batch, wd, gu
    batch.close()
    for lat in lats:
        lat.close()


def _pack_rhs(lat, gu, rhs):
    import torch
    return torch.cat([gu.pack(lat, r, 0) for r in rhs]).contiguous()


def test_batched_khat(small):
    spec, items, batch, wd, gu = small
    ins = [_pack_rhs(it[1], gu, it[2]) for it in items]
    outs = [torch_zeros_like(x) for x in ins]
    batch.wd_batch_mdagm(ins, outs)
    for (dims, a, k, nr), (U, lat, rhs), o in zip(spec, items, outs):
        for r in range(nr):
            got = gu.unpack(lat, o[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh].contiguous(), 0)
            ref = wilson.apply_Khat(U, rhs[r], k)
            assert gu.site_rel_err(got, ref, 0, dims) < 2e-5


def torch_zeros_like(x):
    import torch
    return torch.zeros_like(x)


@pytest.mark.parametrize("use_graph,resid", [(1, 0), (0, 0), (1, 1), (2, 0), (2, 1)],
                         ids=["graph", "eager", "graph-dfresid", "persistent", "persistent-dfresid"])
def test_batched_cg(small, use_graph, resid):
    spec, items, batch, wd, gu = small
    bs = [_pack_rhs(it[1], gu, it[2]) for it in items]
    xs = [torch_zeros_like(b) for b in bs]
    for it in items:
        it[1].wd_set_residual(resid)
    try:
        infos = batch.wd_batch_cg(bs, xs, wd.cg_params(tol=1e-10, prec=wd.F32), use_graph)
    finally:
        for it in items:
            it[1].wd_set_residual(0)
    s = 0
    for (dims, a, k, nr), (U, lat, rhs), x in zip(spec, items, xs):
        for r in range(nr):
            xr = gu.unpack(lat, x[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh].contiguous(), 0)
            res = np.linalg.norm(rhs[r] - wilson.apply_Khat(U, xr, k)) / np.linalg.norm(rhs[r])
            assert res <= 1.01e-10, (dims, r, res, infos[s])
            assert abs(res - infos[s]["true_rel_resid"]) < 1e-12
            # the single-system solver gives the same solution
            xs1 = lat.half_spinor()
            lat.cg_solve(k, gu.pack(lat, rhs[r], 0), xs1, wd.cg_params(tol=1e-10, prec=wd.F32))
            assert gu.rel_norm_err(xr, gu.unpack(lat, xs1, 0)) < 1e-8
            s += 1


@pytest.fixture(scope="module")
def small4():
    """Three uneven lattices with four right-hand sides each and 12-real links:
    every tile shape (one, two or four right-hand sides per thread of the
    batched hop, or the link-staging pipeline) applies."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    spec = [((4, 4, 4, 4), 0.5, 0.12, 4), ((6, 4, 6, 10), 0.4, 0.128, 4), ((8, 8, 8, 8), 0.4, 0.125, 4)]
    stream = torch.cuda.current_stream()
    items = [_make(d, a, k, nr, 1900 + 10 * i, wd, gu, stream, wd.RECON_12) for i, (d, a, k, nr) in enumerate(spec)]
    lats = [it[1] for it in items]
    batch = wd.Batch(lats, [s[2] for s in spec], [s[3] for s in spec])
    yield spec, items, batch, wd, gu
    batch.close()
    for lat in lats:
        lat.close()


SHAPES = [(128, 1, 0), (64, 1, 0), (256, 1, 0), (128, 2, 0), (256, 2, 0), (128, 4, 0), (256, 4, 0), (128, 1, 1)]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{t}x{r}" + ("-staged" if st else "") for t, r, st in SHAPES])
def test_batched_khat_every_tile_shape(small4, shape):
    spec, items, batch, wd, gu = small4
    batch.wd_batch_set_shape(*shape)
    assert batch.wd_batch_shape() == dict(items_per_block=shape[0], rhs_per_thread=shape[1], link_staging=shape[2])
    ins = [_pack_rhs(it[1], gu, it[2]) for it in items]
    outs = [torch_zeros_like(x) for x in ins]
    batch.wd_batch_mdagm(ins, outs)
    for (dims, a, k, nr), (U, lat, rhs), o in zip(spec, items, outs):
        for r in range(nr):
            got = gu.unpack(lat, o[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh].contiguous(), 0)
            assert gu.site_rel_err(got, wilson.apply_Khat(U, rhs[r], k), 0, dims) < 2e-5


@pytest.mark.parametrize("shape,mode", [((128, 2, 0), 1), ((128, 4, 0), 1), ((128, 1, 1), 1), ((128, 1, 0), 2),
                                        ((128, 2, 0), 2), ((64, 4, 0), 2)],
                         ids=["128x2-graph", "128x4-graph", "128x1-staged-graph", "128x1-persistent",
                              "128x2-persistent", "64x4-persistent"])
def test_batched_cg_multi_rhs_per_thread(small4, shape, mode):
    """CG with the stop flags per system: right-hand sides of one thread converge
    at different iterations, so each thread writes only its running systems;
    graph-replayed launches and the persistent cooperative kernel."""
    spec, items, batch, wd, gu = small4
    batch.wd_batch_set_shape(*shape)
    bs = [_pack_rhs(it[1], gu, it[2]) for it in items]
    xs = [torch_zeros_like(b) for b in bs]
    infos = batch.wd_batch_cg(bs, xs, wd.cg_params(tol=1e-10, prec=wd.F32), mode)
    s = 0
    for (dims, a, k, nr), (U, lat, rhs), x in zip(spec, items, xs):
        for r in range(nr):
            xr = gu.unpack(lat, x[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh].contiguous(), 0)
            res = np.linalg.norm(rhs[r] - wilson.apply_Khat(U, xr, k)) / np.linalg.norm(rhs[r])
            assert res <= 1.01e-10, (dims, r, res, infos[s])
            s += 1
    assert len({i["iters"] for i in infos}) > 1       # systems did stop at different iterations


def test_batched_cg_mode_checked(small):
    spec, items, batch, wd, gu = small
    bs = [_pack_rhs(it[1], gu, it[2]) for it in items]
    xs = [torch_zeros_like(b) for b in bs]
    for bad in (-1, 3):
        with pytest.raises(wd.WdError) as e:
            batch.wd_batch_cg(bs, xs, wd.cg_params(tol=1e-10, prec=wd.F32), bad)
        assert e.value.code == 1


def test_batched_shape_arguments_checked(small):
    spec, items, batch, wd, gu = small
    # nrhs 3 and 1 are not multiples of 2; staging needs 12-real links, 128 items, one rhs per thread
    for bad in ((96, 1, 0), (128, 3, 0), (128, 2, 0), (128, 1, 1), (64, 1, 1), (128, 1, 2)):
        with pytest.raises(wd.WdError) as e:
            batch.wd_batch_set_shape(*bad)
        assert e.value.code == 1


@pytest.mark.slow
def test_batched_workload_full_size():
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    work = synthetic.batched_workload()
    stream = torch.cuda.current_stream()
    lats, bs, xs, Us = [], [], [], []
    for i, w in enumerate(work):
        U = synthetic.gauge_field(w["dims"], w["a"], w["seed"])
        lat = wd.Lattice(w["dims"], stream=stream)
        lat.wd_gauge_load(gu.dev(U))
        lat.wd_set_recon(wd.RECON_12)
        b = torch.empty(w["nrhs"] * 24 * lat.Vh, dtype=torch.float64, device="cuda")
        for r in range(w["nrhs"]):
            lat.gaussian_draw(0, 0, w["seed"], 10 + r, b[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh])
        lats.append(lat)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        Us.append(U if i % 8 == 0 else None)
    batch = wd.Batch(lats, [w["kappa"] for w in work], [w["nrhs"] for w in work])
    for mode in (1, 2):                                  # graph-replayed launches; persistent kernel
        for x in xs:
            x.zero_()
        infos = batch.wd_batch_cg(bs, xs, wd.cg_params(tol=1e-10, prec=wd.F32), mode)
        s = 0
        for w, lat, b, x in zip(work, lats, bs, xs):
            for r in range(w["nrhs"]):
                sl = slice(r * 24 * lat.Vh, (r + 1) * 24 * lat.Vh)
                Kx = lat.half_spinor()
                lat.mdagm_apply(w["kappa"], wd.F64, 1, x[sl].contiguous(), Kx)
                rel = float(torch.linalg.vector_norm(b[sl] - Kx) / torch.linalg.vector_norm(b[sl]))
                assert rel <= 1.01e-10, (mode, w["dims"], r, rel, infos[s])
                s += 1
    # batched K_hat against the oracle's sampled sites, one lattice per size,
    # on host-drawn inputs placed in the first right-hand side
    ins = [b.clone() for b in bs]
    psis = {}
    for i in (0, 8, 16):
        dims = work[i]["dims"]
        psis[i] = lattice.mask(synthetic.spinor_field(dims, work[i]["seed"] + 77), dims, 0)
        ins[i][:24 * lats[i].Vh] = gu.pack(lats[i], psis[i], 0)
    outs = [torch.zeros_like(b) for b in bs]
    batch.wd_batch_mdagm(ins, outs)
    rng = np.random.default_rng(3)
    for i in (0, 8, 16):
        w, lat = work[i], lats[i]
        dims = w["dims"]
        psi = psis[i]
        got = gu.unpack(lat, outs[i][:24 * lat.Vh].contiguous(), 0).reshape(-1, 4, 3)
        par = lattice.parity(dims).reshape(-1)
        idx = np.sort(rng.choice(np.flatnonzero(par == 0), 64, replace=False))
        ref = sampled.khat_at(Us[i], psi, w["kappa"], idx)
        d = np.sqrt(np.sum(np.abs(got[idx] - ref) ** 2, axis=(-2, -1)))
        rr = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-2, -1)))
        assert np.max(d / rr) < 4e-5
    info = batch.wd_batch_info()
    assert info["systems"] == 96
    batch.close()
    for lat in lats:
        lat.close()
