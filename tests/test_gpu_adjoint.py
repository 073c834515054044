"""Exact gradients and Newton refinement at peaks (fc2_backward), against the
oracle's analytic gradients, central finite differences of the oracle's
Delta chi^2, and its Brent maximum."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


def test_backward_matches_oracle_and_fd(fc2, oracle_mod):
    c = synth.short_curve(n=600, N=8192)
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed", top_k=4) as p:
        _, best, peaks, chi0 = p.execute()
        js = np.array([q["j"] for q in peaks])
        g = np.array([1.0, -0.5, 2.0, 0.25])
        r = p.backward(js, grad_out=g)
    H = c.H
    for k, j in enumerate(js):
        f = c.f_min + j * c.df
        d, gf, gx, gs = oracle_mod.grad(c.t, c.x, c.sigma, H, f)
        assert r["d_df"][k] == pytest.approx(g[k] * gf, rel=1e-7, abs=1e-9 * abs(gf) + 1e-12)
        np.testing.assert_allclose(r["d_dx"][k], g[k] * gx, rtol=1e-7, atol=1e-9 * np.abs(gx).max())
        np.testing.assert_allclose(r["d_dsigma"][k], g[k] * gs, rtol=1e-7, atol=1e-9 * np.abs(gs).max())
        # central differences of the exact Delta chi^2 (the oracle's)
        D = lambda xx, ss, ff: oracle_mod.dchi2_freqs(c.t, xx, ss, H, [ff], threads=1)[0, H - 1]  # noqa
        hf = 1e-7 / (c.t.max() - c.t.min())
        fd = (D(c.x, c.sigma, f + hf) - D(c.x, c.sigma, f - hf)) / (2 * hf)
        assert r["d_df"][k] / g[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(d) * 100)
        for i in (0, 123, 377):
            h = 1e-6 * c.sigma[i]
            xp, xm = c.x.copy(), c.x.copy()
            xp[i] += h
            xm[i] -= h
            fdx = (D(xp, c.sigma, f) - D(xm, c.sigma, f)) / (2 * h)
            assert r["d_dx"][k][i] / g[k] == pytest.approx(fdx, rel=1e-5, abs=1e-8 * abs(d) / c.sigma[i])
            sp, sm = c.sigma.copy(), c.sigma.copy()
            sp[i] += h
            sm[i] -= h
            fds = (D(c.x, sp, f) - D(c.x, sm, f)) / (2 * h)
            assert r["d_dsigma"][k][i] / g[k] == pytest.approx(fds, rel=1e-5, abs=1e-8 * abs(d) / c.sigma[i])
        # Newton maximum vs Brent on the same bracket
        fs, vs = oracle_mod.refine(c.t, c.x, c.sigma, H, f - c.df, f + c.df, tol=1e-12)
        assert abs(r["f_refined"][k] - fs) <= 1e-9
        assert r["dchi2_refined"][k] == pytest.approx(vs, rel=1e-9)


def test_backward_unsorted_input_caller_order(fc2, oracle_mod):
    c = synth.short_curve(n=300, N=4096)
    perm = np.random.default_rng(2).permutation(c.n)
    t, x, s = c.t[perm], c.x[perm], c.sigma[perm]
    with fc2.Plan(t, x, s, c.H, c.f_min, c.df, c.N, 2, "fp64", top_k=2) as p:
        _, best, peaks, _ = p.execute()
        j = best[-1]["j"]
        r = p.backward([j])
    _, gf, gx, gs = oracle_mod.grad(t, x, s, c.H, c.f_min + j * c.df)
    np.testing.assert_allclose(r["d_dx"][0], gx, rtol=1e-7, atol=1e-9 * np.abs(gx).max())
    np.testing.assert_allclose(r["d_dsigma"][0], gs, rtol=1e-7, atol=1e-9 * np.abs(gs).max())


def test_backward_batched(fc2, oracle_mod):
    b = synth.adjoint_batch(C=12, n=400, N=1 << 16)
    out, peaks, _ = fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N,
                                        2, "mixed", top_k=3)
    pj = np.array([[q["j"] for q in pk] for pk in peaks])
    r = fc2.backward_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N, pj)
    K = pj.shape[1]
    for c in (0, 5, 11):
        cur = b.curve(c)
        n = cur.n
        for k in range(K):
            f = cur.f_min + pj[c, k] * cur.df
            _, gf, gx, gs = oracle_mod.grad(cur.t, cur.x, cur.sigma, cur.H, f)
            o = K * int(b.offsets[c]) + k * n
            np.testing.assert_allclose(r["d_dx"][o:o + n], gx, rtol=1e-7, atol=1e-9 * np.abs(gx).max())
            np.testing.assert_allclose(r["d_dsigma"][o:o + n], gs, rtol=1e-7, atol=1e-9 * np.abs(gs).max())
            assert r["d_df"][c, k] == pytest.approx(gf, rel=1e-7, abs=1e-9 * abs(gf) + 1e-12)
            # the local maximum next to the bin (the grid is fine enough that it
            # lies within half a bin of the bin's centre)
            fs, vs = oracle_mod.refine(cur.t, cur.x, cur.sigma, cur.H, f - 0.5 * cur.df,
                                       f + 0.5 * cur.df, tol=1e-12)
            assert abs(r["f_refined"][c, k] - fs) <= 1e-9
            assert r["dchi2_refined"][c, k] == pytest.approx(vs, rel=1e-9)


def test_autograd_function(fc2):
    import torch
    c = synth.short_curve(n=200, N=2048)
    F = fc2.peaks_function()
    x = torch.tensor(c.x, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(c.sigma, dtype=torch.float64, requires_grad=True)
    vals, js = F.apply(x, s, c.t, c.H, c.f_min, c.df, c.N, 2, "fp64", 3)
    (vals * torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64)).sum().backward()
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "fp64", top_k=3) as p:
        r = p.backward(js.numpy(), grad_out=[1.0, 2.0, 3.0])
    np.testing.assert_allclose(x.grad.numpy(), r["d_dx"].sum(0), rtol=1e-12)
    np.testing.assert_allclose(s.grad.numpy(), r["d_dsigma"].sum(0), rtol=1e-12)
