"""Learned rank predictor end to end on the GPU: ranks recorded by the
factorization on the small and batched workloads train the network with the
library's own kernels; on held-out problems it must beat the best constant
predictor clearly, and the learned mixed form (the prediction gates the
precision of each cluster's compression) must keep the mixed form's bars
against FP64: iterations within 1, true residual <= 1e-8, at most 5% of
ranks differing; no cluster the rank-0 certificate accepts has a nonzero
rank in FP64.  The same bars hold on the 512x512x20 workload."""
import numpy as np
import pytest

from paper_1811_11248_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_1811_11248_gb300 import build, hsolve, rank_model
    build.build()
    hsolve.lib()
    f1, r1, s1 = rank_model.collect(inputs.anisotropic_16x16x8(), depth=4)
    f3, r3, s3 = rank_model.collect_batched([inputs.batched_problem(k) for k in range(24)])
    X = np.concatenate([f1, f3])
    R = np.concatenate([r1, r3])
    S = np.concatenate([s1, s3])
    model, losses = rank_model.fit(X, R, S, epochs=30)
    return hsolve, rank_model, model, losses


def test_training_converges(trained):
    _, _, _, losses = trained
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.2 * losses[:10].mean()


def test_prediction_beats_constant_on_held_out(trained):
    _, rank_model, model, _ = trained
    f, r, s = rank_model.collect_batched([inputs.batched_problem(k) for k in range(240, 256)])
    acc = rank_model.accuracy(model, f, r, s)
    print("held-out batched problems:", acc)
    assert acc["mae"] <= 0.6 * acc["mae_constant"]
    assert acc["exact"] >= 0.6


def test_learned_mixed_form(trained):
    hs, rank_model, model, _ = trained
    p = inputs.grid_operator(32, 32, 16, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
    st = torch.cuda.current_stream().cuda_stream

    def run(precision, model_vec):
        opt = hs.hs_default_options(tol=1e-2, mem=hs.HS_MEM_HOST, coords=p.coords, stream=st, precision=precision,
                                    rank_model=model_vec, profile=1)
        h = hs.hs_setup(p.n, p.rowptr, p.col, p.val, opt=opt)
        x = torch.empty(p.n, dtype=torch.float64, device="cuda")
        info, rc = h.hs_krylov(torch.from_numpy(p.b).cuda(), x)
        ranks = np.concatenate([h.level_info(l)[1] for l in range(h.num_levels())])
        stats = h.kernel_stats()
        h.close()
        return info, x.cpu().numpy(), ranks, stats

    i64, _, r64, _ = run(hs.HS_PREC_FP64, None)
    imx, _, rmx, smx = run(hs.HS_PREC_MIXED, None)
    ilr, xlr, rlr, slr = run(hs.HS_PREC_MIXED, model.packed())
    res = np.linalg.norm(p.b - p.matvec(xlr)) / np.linalg.norm(p.b)
    print(f"iterations fp64 {i64.iters} mixed {imx.iters} learned {ilr.iters}; factor ms mixed "
          f"{smx['factor']['ms']:.3f} learned {slr['factor']['ms']:.3f}; ranks differing from fp64: "
          f"mixed {int(np.sum(rmx != r64))} learned {int(np.sum(rlr != r64))} of {len(r64)}")
    assert res <= 1e-8 and ilr.rel_resid <= 1e-8
    assert abs(ilr.iters - i64.iters) <= 1
    assert np.sum(rlr != r64) <= 0.05 * len(r64)
    # the rank-0 certificate proves ||G^-1 A_sw||_F <= eps: a cluster it
    # certifies (rank 0 here, above 0 without the predictor) has rank 0 in FP64
    certified = (rlr == 0) & (rmx > 0)
    print(f"certified rank 0 where the mixed form's QR found a rank: {int(certified.sum())}")
    assert np.sum(certified & (r64 > 0)) == 0


@pytest.mark.slow
def test_learned_form_at_512x512x20(trained):
    """The predictor trained as the benchmark trains it (ranks of the 16x16x8,
    64x64x16 and batched 0-63 workloads) on the 512x512x20 workload: the
    learned mixed form keeps the mixed form's iterations (within 1) and
    residual, and at most 5% of its ranks differ from the mixed form's.  Its
    factor time is printed; the time gained is measured by the benchmark
    (several timed samples per form), not asserted here."""
    hs, rank_model, _, _ = trained
    f1, r1, s1 = rank_model.collect(inputs.anisotropic_16x16x8(), depth=4)
    f2, r2, s2 = rank_model.collect(inputs.anisotropic_64x64x16(), depth=8)
    f3, r3, s3 = rank_model.collect_batched([inputs.batched_problem(k) for k in range(64)])
    model, _ = rank_model.fit(np.concatenate([f1, f2, f3]), np.concatenate([r1, r2, r3]),
                              np.concatenate([s1, s2, s3]), epochs=40)
    p = inputs.anisotropic_512x512x20()
    st = torch.cuda.current_stream().cuda_stream
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, va, b = dev(p.rowptr), dev(p.col), dev(p.val), dev(p.b)
    coords = np.ascontiguousarray(p.coords)
    res = {}
    for name, mv in (("mixed", None), ("learned", model.packed())):
        opt = hs.hs_default_options(tol=1e-2, rtol=1e-8, mem=hs.HS_MEM_DEVICE, stream=st, coords=coords,
                                    precision=hs.HS_PREC_MIXED, rank_model=mv, profile=1)
        h = hs.hs_setup(p.n, rp, ci, va, opt=opt)
        x = torch.empty(p.n, dtype=torch.float64, device="cuda")
        info, rc = h.hs_krylov(b, x)
        ranks = np.concatenate([h.level_info(l)[1] for l in range(h.num_levels())])
        res[name] = (h.kernel_stats()["factor"]["ms"], info.iters, info.rel_resid, ranks)
        h.close()
    print("factor ms and iterations:", {k: v[:3] for k, v in res.items()})
    # clusters certified rank 0 where the mixed form's FP32 QR found a rank:
    # only threshold cases (the FP32 QR rounding a norm just below eps above it)
    cert = int(np.sum((res["learned"][3] == 0) & (res["mixed"][3] > 0)))
    print("certified rank 0 where the mixed form's QR found a rank:", cert)
    assert cert <= max(2, 1e-4 * len(res["mixed"][3]))
    assert abs(res["learned"][1] - res["mixed"][1]) <= 1
    assert res["learned"][2] <= 1e-8
    assert np.sum(res["learned"][3] != res["mixed"][3]) <= 0.05 * len(res["mixed"][3])
