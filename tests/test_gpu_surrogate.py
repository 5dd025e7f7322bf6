"""The learned surrogate on the GPU: its BF16/FP32 GEMM in every storage
order, its loss and gradients against the FP64 oracle (oracle/surrogate.py),
and the whole workflow on a small model -- solver catalog, training on the
GPU, error gate, serving with the solver as fallback -- where every served
seismogram is checked against the exact solver reference."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es, surrogate
    es._load()
    return es, surrogate, torch


def _bf(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


@pytest.mark.parametrize("a_t", [False, True])
@pytest.mark.parametrize("b_nk", [False, True])
@pytest.mark.parametrize("split", [1, 3])
def test_gemm_all_layouts(env, a_t, b_nk, split):
    es, sur, torch = env
    rng = np.random.default_rng(int(a_t) * 4 + int(b_nk) * 2 + split)
    M, N, K = 200, 136, 328  # ragged against the 128 x 128 x 32 tiles
    A = rng.standard_normal((K, M) if a_t else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if b_nk else (K, N)).astype(np.float32)
    Ab, Bb = _bf(torch, A), _bf(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)  # the BF16-rounded operands
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    opA = A64.T if a_t else A64
    opB = B64.T if b_nk else B64
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    sur.es_gemm_bf16(Ab, Bb, C, a_t=a_t, b_nk=b_nk, alpha=0.5, beta=-2.0, split_k=split)
    ref = 0.5 * opA @ opB - 2.0 * C0
    got = C.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("M,N,K,split,beta", [(8, 8, 8, 1, 0.0), (128, 256, 64, 1, 0.0), (300, 520, 1000, 1, 1.5),
                                               (256, 1000, 4608, 6, -0.5), (130, 260, 136, 1, 0.0),
                                               (64, 4608, 8192, 16, 0.0), (2000, 4000, 200, 1, 0.5),
                                               (4096, 8192, 64, 1, 0.0)])
def test_tcgen05_gemm_k_major(env, M, N, K, split, beta):
    """Both operands K-major: the persistent tcgen05 kernel (TMA ring, two
    tensor-memory accumulators), single tiles, ragged edges in M, N and K,
    split-K, and grids of 256 and 1024 tiles (several per CTA)."""
    import ctypes
    es, sur, torch = env
    rng = np.random.default_rng(M + N + K + split)
    lda, ldb, ldc = K + 8, K + 16, N + 4  # leading dimensions past the matrix edge
    A = rng.standard_normal((M, lda)).astype(np.float32)
    B = rng.standard_normal((N, ldb)).astype(np.float32)
    Ab, Bb = _bf(torch, A), _bf(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)[:, :K]
    B64 = Bb.float().cpu().numpy().astype(np.float64)[:, :K]
    C0 = rng.standard_normal((M, ldc)).astype(np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = sur._lib().es_gemm_bf16(M, N, K, vp(Ab), lda, 0, vp(Bb), ldb, 1, vp(C), ldc, ctypes.c_float(0.75),
                                 ctypes.c_float(beta), split, None)
    assert rc == 0
    sur.es_gemm_status()
    ref = 0.75 * A64 @ B64.T + beta * C0[:, :N]
    got = C.cpu().numpy()
    assert np.abs(got[:, :N] - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.array_equal(got[:, N:], C0[:, N:])  # columns past N untouched


def test_bounded_wait_times_out_and_the_context_survives(env):
    """The failure path of the tcgen05 GEMM's bounded waits, without a fault
    or a hang: a wait on a barrier phase that nothing completes gives up after
    50 ms, the status word reports ES_ERR_TIMEOUT once and is cleared, and the
    same context then runs a tcgen05 GEMM correctly."""
    import time
    es, sur, torch = env
    sur.es_gemm_status()  # starts clear
    t0 = time.perf_counter()
    sur.es_gemm_wait_probe(0.05)
    with pytest.raises(es.EsError) as err:
        sur.es_gemm_status()
    assert err.value.status == es.ES_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.05
    sur.es_gemm_status()  # read once, then clear
    rng = np.random.default_rng(1)
    A, B = _bf(torch, rng.standard_normal((136, 200))), _bf(torch, rng.standard_normal((264, 200)))
    C = torch.zeros((136, 264), device="cuda")
    sur.es_gemm_bf16(A, B, C, b_nk=True)
    sur.es_gemm_status()
    ref = A.float().cpu().numpy().astype(np.float64) @ B.float().cpu().numpy().astype(np.float64).T
    assert np.abs(C.cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max()


def test_loss_and_gradients_match_oracle(env):
    es, sur, torch = env
    from oracle import surrogate as osur
    cfg = dict(nfreq=2, hidden=64, latent=16, n_rcv=4, nt=16)
    s = sur.Surrogate(cfg["n_rcv"], cfg["nt"], nfreq=2, hidden=64, latent=16, max_batch=16, seed=3)
    try:
        rng = np.random.default_rng(5)
        lay, P, F, D = osur.layout(**cfg)
        assert s.num_params() == P
        params = (rng.standard_normal(P) * 0.2).astype(np.float32)
        s.set_params(params)
        scale = [1.5, 0.7, 0.9, 1.1]
        s.set_output_scale(scale)
        B = 16
        pos = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
        mt = rng.standard_normal((B, 6)).astype(np.float32)
        tgt = rng.standard_normal((B, D)).astype(np.float32)
        cu = lambda a: torch.from_numpy(a).cuda()
        loss, per, g = s.loss_grad(cu(pos), cu(mt), cu(tgt))
        # the oracle sees the parameters the GPU multiplies with (BF16-rounded weights)
        pb = torch.from_numpy(params).to(torch.bfloat16).float().numpy().astype(np.float64)
        pr = params.astype(np.float64).copy()
        for name in ("W1", "W2", "W3", "Wd"):
            o, shp = lay[name]
            pr[o:o + int(np.prod(shp))] = pb[o:o + int(np.prod(shp))]
        oloss, oper, og = osur.loss_and_grads(pr, cfg, pos, mt, tgt, scale)
        assert abs(loss - oloss) <= 2e-2 * oloss
        assert np.allclose(per.cpu().numpy(), oper, rtol=3e-2)
        g = g.cpu().numpy().astype(np.float64)
        # BF16 operands round to 2^-9 relative; the gradient of the first layer
        # sits behind five such roundings (dU, dA, dH2, dH1, x), the others behind fewer
        tol = {"W1": 6e-2, "b1": 6e-2}
        for name, (o, shp) in lay.items():
            n = int(np.prod(shp))
            a, b = g[o:o + n], og[o:o + n]
            assert np.linalg.norm(a - b) <= tol.get(name, 3e-2) * np.linalg.norm(b), name
        y = s.predict(cu(pos), cu(mt)).cpu().numpy()
        assert np.linalg.norm(y - osur.forward(pr, cfg, pos, mt, scale)["Y"]) <= 1e-2 * np.linalg.norm(y)
    finally:
        s.close()


def test_train_step_matches_oracle_adam(env):
    """One train step against the oracle's Adam step taken from its own FP64
    gradient (BF16-rounded weights).  The first Adam step moves a parameter by
    lr g / (|g| + eps), so wherever the gradient's sign is certain the GPU's
    update must equal the oracle's to FP32 rounding, and no parameter may move
    by more than lr.  The decoder has 96 rows (ragged 64-row tiles of the
    fused step).  Then predict() must run on the updated decoder: its K-major
    copy is refreshed by the step itself."""
    es, sur, torch = env
    from oracle import surrogate as osur
    cfg = dict(nfreq=2, hidden=64, latent=16, n_rcv=4, nt=16)
    s = sur.Surrogate(cfg["n_rcv"], cfg["nt"], nfreq=2, hidden=64, latent=16, max_batch=16, seed=3)
    try:
        rng = np.random.default_rng(11)
        lay, P, F, D = osur.layout(**cfg)
        params = (rng.standard_normal(P) * 0.2).astype(np.float32)
        s.set_params(params)
        scale = [1.5, 0.7, 0.9, 1.1]
        s.set_output_scale(scale)
        B, lr = 16, 2e-2
        pos = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
        mt = rng.standard_normal((B, 6)).astype(np.float32)
        tgt = rng.standard_normal((B, D)).astype(np.float32)
        cu = lambda a: torch.from_numpy(a).cuda()
        s.predict(cu(pos), cu(mt))  # the K-major copy of the initial decoder exists before the step
        s.train_step(cu(pos), cu(mt), cu(tgt), lr)
        after = s.get_params().astype(np.float64)

        def bf16(x):
            out = np.asarray(x, np.float64).copy()
            r = torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()
            for name in ("W1", "W2", "W3", "Wd"):
                o, shp = lay[name]
                out[o:o + int(np.prod(shp))] = r[o:o + int(np.prod(shp))]
            return out

        _, _, og = osur.loss_and_grads(bf16(params), cfg, pos, mt, tgt, scale)
        exp, _, _ = osur.adam_step(params.astype(np.float64), og, 0.0, 0.0, 1, lr)
        moved = after - params.astype(np.float64)
        assert np.abs(moved).max() <= lr * (1 + 1e-3)
        # The GPU's gradient is within tol * |g| of the oracle's (the bound of the gradient test), so
        # an element larger than that keeps its sign and must take the oracle's step exactly; below
        # it BF16 rounding may flip a sign, which at most 5 % of the elements may show.
        tol = {"W1": 6e-2, "b1": 6e-2}
        for name, (o, shp) in lay.items():
            n = int(np.prod(shp))
            g = og[o:o + n]
            dev = np.abs(after[o:o + n] - exp[o:o + n])
            sure = np.abs(g) > tol.get(name, 3e-2) * np.linalg.norm(g)
            assert not sure.any() or dev[sure].max() <= 1e-3 * lr, name
            nz = g != 0
            assert np.mean(dev[nz] <= 1e-3 * lr) >= 0.95, (name, np.mean(dev[nz] <= 1e-3 * lr))
        y = s.predict(cu(pos), cu(mt)).cpu().numpy()
        ref = osur.forward(bf16(after.astype(np.float32)), cfg, pos, mt, scale)["Y"]
        stale = osur.forward(bf16(np.concatenate([after[:lay["Wd"][0]], params[lay["Wd"][0]:]]).astype(np.float32)),
                             cfg, pos, mt, scale)["Y"]
        assert np.linalg.norm(ref - stale) > 5e-2 * np.linalg.norm(ref)  # the step moved the decoder visibly
        assert np.linalg.norm(y - ref) <= 1e-2 * np.linalg.norm(ref)
    finally:
        s.close()


@pytest.mark.parametrize("n_src", [40, 37])
def test_serve_trusted_sources(env, n_src):
    """Every location trusted: serve() predicts runs of consecutive sources
    straight into the caller's buffer (a ragged tail through a padded batch);
    the result equals predict() on the same inputs, bit for bit."""
    es, sur, torch = env
    s = sur.Surrogate(2, 16, nfreq=2, hidden=32, latent=8, max_batch=16, seed=2)
    try:
        rng = np.random.default_rng(n_src)
        pos_n = rng.uniform(-1, 1, (5, 3)).astype(np.float32)
        loc = rng.integers(0, 5, n_src)
        mts = rng.standard_normal((n_src, 6))
        buf = torch.full((n_src, 4, 2, 16), float("nan"), device="cuda")
        out, used = sur.serve(s, pos_n, np.ones(5, bool), loc, mts, None, None, 16, 0.0, np.zeros((2, 3), np.int32),
                              None, out=buf)
        assert out.data_ptr() == buf.data_ptr() and not used.any()
        for b in range(0, n_src, 16):
            n = min(16, n_src - b)
            k = (n + 7) // 8 * 8
            idx = np.concatenate([np.arange(b, b + n), np.full(k - n, b)])
            ref = s.predict(torch.from_numpy(pos_n[loc[idx]]).cuda(),
                            torch.from_numpy(mts[idx].astype(np.float32)).cuda())[:n]
            assert torch.equal(out[b:b + n].reshape(n, -1), ref), b
    finally:
        s.close()


def test_catalog_train_gate_serve(env):
    """Small marine model, 24 catalog locations: the surrogate learns their
    Green's functions from 144 solver runs (unit moment tensors), is trained
    on fresh random moment tensors every epoch, the gate keeps the locations it
    reproduces within 5 %, and every served seismogram (surrogate or solver)
    is within 5 % of the exact reference."""
    es, sur, torch = env
    shape = (48, 32, 32)
    rho, cp, cs = synth.marine_model(shape=shape, seed=4)
    pml, nt = 4, 256  # long enough for the full arrivals at every receiver
    dt = cfl_dt(cp, 10.0)
    wav = synth.ricker(nt, dt, 30.0)
    box = synth.reservoir_box(shape, pml)
    rng = synth.SplitMix64(6)
    locations = synth.latin_hypercube_positions(rng, box, 24)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(2, 2)
        G = sur.green_catalog(m, locations, nt, dt, rcv, wav, per_batch=8)
        pos_n = sur.normalize_positions(locations, box)
        s = sur.Surrogate(len(rcv), nt, nfreq=3, hidden=128, latent=64, max_batch=48, seed=1)
        try:
            hist = sur.train(s, pos_n, G, epochs=200, lr=3e-3)
            assert hist[-1] < 1e-4 * hist[0]
            trusted, errs = sur.calibrate_gate(s, pos_n, G, n_val=3)
            assert trusted.mean() >= 0.75, errs.max(axis=1)
            # serve random sources at catalog locations
            loc = np.floor(synth.SplitMix64(9).uniform(40) * len(locations)).astype(int)
            mts = np.array([synth.random_dc(rng) for _ in loc])
            out, used_solver = sur.serve(s, pos_n, trusted, loc, mts, m, locations, nt, dt, rcv, wav)
            ref = sur.combine(G, loc, mts)
            # whole-seismogram relative L2 with each component divided by its RMS over the catalog
            sc = G.permute(2, 0, 1, 3, 4).reshape(4, -1).pow(2).mean(dim=1).sqrt().view(1, 4, 1, 1)
            d = ((out - ref) / sc).reshape(len(loc), -1).norm(dim=1) / (ref / sc).reshape(len(loc), -1).norm(dim=1)
            assert float(d.max()) < 0.05, float(d.max())
            assert used_solver.sum() == (~trusted[loc]).sum()
        finally:
            s.close()


def test_sources_away_from_the_catalog(env):
    """Sources at cells that are not catalog locations: their exact references
    come from fresh solver runs; the network is compared with the two baselines
    without one (the nearest catalog location, inverse-distance interpolation
    of the catalog); the position gate, calibrated on held-out cells, decides
    which of them the network may serve.  Every served seismogram -- network
    or solver fallback -- is within 5 % of its exact reference, and the
    fallback runs for the off-catalog sources the gate refuses."""
    es, sur, torch = env
    shape = (48, 32, 32)
    rho, cp, cs = synth.marine_model(shape=shape, seed=4)
    pml, nt = 4, 256
    dt = cfl_dt(cp, 10.0)
    wav = synth.ricker(nt, dt, 30.0)
    box = synth.reservoir_box(shape, pml)
    rng = synth.SplitMix64(6)
    locations = synth.latin_hypercube_positions(rng, box, 24)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(2, 2)
        G = sur.green_catalog(m, locations, nt, dt, rcv, wav, per_batch=8)
        sc = sur.component_scale(G)
        s = sur.Surrogate(len(rcv), nt, nfreq=3, hidden=128, latent=64, max_batch=48, seed=1)
        try:
            sur.train(s, sur.normalize_positions(locations, box), G, epochs=200, lr=3e-3)
            trusted, _ = sur.calibrate_gate(s, sur.normalize_positions(locations, box), G, n_val=3)
            # held-out cells off the catalog
            cand = synth.random_positions(synth.SplitMix64(12), box, 64)
            _, dc = sur.nearest_locations(locations, cand)
            held = cand[dc[:, 0] > 0][:16]
            hmt = np.array([synth.random_dc(rng) for _ in held])
            truth = sur.solver_references(m, held, hmt, nt, dt, rcv, wav)
            _, hd = sur.nearest_locations(locations, held)
            e_net = sur.scaled_rel_l2(sur.predict_at(s, box, held, hmt), truth, sc)
            e_near = sur.scaled_rel_l2(sur.baseline_nearest(G, locations, held, hmt), truth, sc)
            e_idw = sur.scaled_rel_l2(sur.baseline_idw(G, locations, held, hmt), truth, sc)
            assert np.isfinite(e_net).all() and np.isfinite(e_near).all() and np.isfinite(e_idw).all()
            print(f"off-catalog: within 5 % {np.mean(e_net < 0.05):.3f}; median error network {np.median(e_net):.3f}, "
                  f"nearest location {np.median(e_near):.3f}, inverse-distance {np.median(e_idw):.3f}")
            d_star = sur.calibrate_position_gate(hd[:, 0], e_net)
            # a mix of catalog and off-catalog sources, not the held-out ones
            pos = np.concatenate([locations[:8], cand[dc[:, 0] > 0][16:24]])
            mts = np.array([synth.random_dc(rng) for _ in pos])
            out, used = sur.serve_positions(s, box, trusted, d_star, locations, pos, mts, m, nt, dt, rcv, wav)
            ref = sur.solver_references(m, pos, mts, nt, dt, rcv, wav)
            err = sur.scaled_rel_l2(out, ref, sc)
            assert err.max() < 0.05, err
            _, pd = sur.nearest_locations(locations, pos)
            assert used[pd[:, 0] > max(d_star, 0)].all()  # beyond the gate's distance: the solver
            assert used.any() and (~used[:8]).sum() == trusted[:8].sum()
        finally:
            s.close()
