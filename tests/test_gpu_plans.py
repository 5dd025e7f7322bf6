"""Every candidate FFT plan (radix order R1 x R2) computes the same staggered
derivative as the oracle, and the autotuner times the candidates on a
model's own passes, keeps one of them and records it in the plan cache."""
import numpy as np
import pytest

from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def es():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es as _es
    _es._load()
    yield _es
    for n, cands in _es.PLAN_CANDIDATES.items():  # back to the defaults
        for kind in (0, 1):
            _es.es_fft_plan_select(kind, n, *cands[0])


@pytest.mark.parametrize("n", [32, 48, 64, 75, 80, 96, 125, 128, 160, 192])
def test_every_plan_matches_oracle(es, orc, n):
    """Along x, and along y and z with an even and an odd nx (the y / z passes
    move pencil pairs as float2 or, for an odd nx, as two floats)."""
    import torch
    rng = np.random.default_rng(n)
    for axis, shape in ((0, (16, 32, n)), (1, (16, n, 32)), (2, (n, 16, 32)), (1, (16, n, 33)),
                        (2, (n, 16, 45))):
        f = rng.standard_normal(shape).astype(np.float32)
        ref = orc.deriv(f.astype(np.float64), axis, 10.0, +1)
        kind = 0 if axis == 0 else 1
        for ra, rb in es.PLAN_CANDIDATES[n]:
            es.es_fft_plan_select(kind, n, ra, rb)
            assert es.es_fft_plan(kind, n) == (ra, rb)
            out = torch.empty(shape, device="cuda")
            es.es_derivative(torch.from_numpy(f).cuda(), axis, 10.0, +1, out)
            got = out.cpu().numpy().astype(np.float64)
            assert rel_l2(got, ref) < 2e-6, (axis, ra, rb)
        es.es_fft_plan_select(kind, n, *es.PLAN_CANDIDATES[n][0])


def test_autotune_picks_a_candidate_and_caches_it(es, tmp_path, monkeypatch):
    from paper_1705_04874_gb300 import synth
    cache = tmp_path / "plans.txt"
    monkeypatch.setenv("ES_TUNE_CACHE", str(cache))
    rho, cp, cs = synth.marine_model(shape=(160, 96, 128), seed=2)
    with es.Model(rho, cp, cs, dx=10.0, pml=8) as m:
        report = m.autotune(reps=3)
        assert es.es_fft_plan(0, 128) in es.PLAN_CANDIDATES[128]
        assert es.es_fft_plan(1, 96) in es.PLAN_CANDIDATES[96]
        assert es.es_fft_plan(1, 160) in es.PLAN_CANDIDATES[160]
        assert np.all(m.state_get() == 0)
    lines = [l for l in report.splitlines() if l.strip()]
    assert len(lines) == 2 + 2 + 2  # two candidates each for x=128, y=96, z=160
    text = cache.read_text().splitlines()
    assert len(text) == 3 and all(l.count("|") == 4 for l in text)
