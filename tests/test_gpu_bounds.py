"""The bounds-checked debug build (libes_bounds.so, -DES_BOUNDS=1): in a
process of its own (ES_BOUNDS=1), runs through every kind of derivative pass
-- even and odd lengths, two- and three-stage plans, odd nx, circulant and
tensor-core axes, compensated passes, batches with an odd cell count, fused
sources and receivers, the stand-alone derivative and Laplacian -- record no
index out of range, and the runs still match the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + '/tests')
from paper_1705_04874_gb300 import es, synth
import oracle as orc
from conftest import cfl_dt, trace_errors, rel_l2
assert es.bounds_build() and es.library_path().endswith('libes_bounds.so')
out = {}

def bad():
    return es.es_debug_bounds()[2]

def run(shape, pml, nt, prec=0, nb=1, oracle=True, seed=1, d=(10.0, 10.0, 10.0)):
    rho, cp, cs = synth.marine_model(shape=shape, seed=seed)
    dt = cfl_dt(cp, min(d))
    w = synth.ricker(nt, dt, 30.0)
    rng = synth.SplitMix64(seed)
    pos = synth.random_positions(rng, synth.reservoir_box(shape, pml), nb)
    mts = np.array([synth.explosive() for _ in range(nb)])
    rcv = orc.seabed_receivers(cs, pml, 3, 3)
    with es.Model(rho, cp, cs, dx=d[0], pml=pml) as m:
        if d[1] != d[0] or d[2] != d[0]:
            m.set_spacing(*d)
        m.set_precision(prec)
        if nb == 1:
            m.source_set(pos[0], mts[0], w)
        else:
            m.batch_set(pos, mts, np.stack([w] * nb))
        tr = m.run(nt, dt, rcv)
    res = {'bad': bad()}
    if oracle:
        ref = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=pml,
                           sources=[dict(kind='moment', pos=pos[0], m=mts[0], w=w)], receivers=rcv)['traces']
        res['err'] = float(trace_errors(tr if nb == 1 else tr[0], ref).max())
    return res

out['fft_even'] = run((32, 32, 48), 5, 60)
out['fft_odd_nx'] = run((48, 32, 75), 5, 60, d=(12.5, 12.5, 10.0))
out['fft_three_stage'] = run((32, 75, 125), 6, 40, d=(12.5, 12.5, 10.0))
out['batch_odd_cells'] = run((125, 75, 75), 5, 20, nb=3, oracle=False)
out['circulant'] = run((27, 30, 33), 4, 60)
out['compensated'] = run((24, 20, 32), 4, 40, prec=es.ES_PREC_COMPENSATED)
out['tensor_core'] = run((193, 12, 20), 3, 30, prec=es.ES_PREC_FP32_TC)
for shape in ((7, 5, 125), (16, 75, 33), (75, 16, 48)):
    f = torch.randn(shape, device='cuda')
    o = torch.empty_like(f)
    for axis in range(3):
        es.es_derivative(f, axis, 10.0, 1, o)
out['derivative'] = {'bad': bad()}
for shape in ((301, 75, 125), (30, 48, 40)):
    f = torch.randn(shape, device='cuda')
    o = torch.empty_like(f)
    es.es_laplacian(f, (12.5, 12.5, 10.0), o)
out['laplacian'] = {'bad': bad()}
print('RESULT ' + json.dumps(out))
"""


def test_bounds_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, ES_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    for case, v in res.items():
        assert v["bad"] == 0, (case, v["bad"] >> 40, v["bad"] & ((1 << 40) - 1))
        if "err" in v:
            assert v["err"] < 1e-4, (case, v["err"])
