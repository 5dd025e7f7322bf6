"""The learned surrogate (include/es_surrogate.h): ctypes binding plus the
workflow around it -- a catalog of source locations whose unit-moment-tensor
responses come from the solver, training, an error gate calibrated on
held-out moment tensors, and serving with the solver as the fallback.

The paper (Sec. III-A, VI-A) simulates single sources at a catalog of Latin-
hypercube locations and builds every multi-event scenario from those traces;
it names a learned proxy of the forward simulation as future work
(Sec. VII-C).  Here the network learns the catalog's Green's functions: for a
location p and moment tensor M the traces are sum_c M_c G_c(p) (exact
linearity of the elastic equations), the network predicts them as
(M (x) a(p)) Wd, and the solver produces every training target and every
reference.  All arithmetic runs in the library's kernels; this module only
moves pointers, picks batches and keeps the bookkeeping.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import es as _es
from . import synth


class Config(ctypes.Structure):
    _fields_ = [("nfreq", ctypes.c_int), ("hidden", ctypes.c_int), ("latent", ctypes.c_int),
                ("n_rcv", ctypes.c_int), ("nt", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("seed", ctypes.c_ulonglong)]


_bound = False


def _lib():
    global _bound
    lib = _es._load()
    if not _bound:
        vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        sig = {
            "es_sur_create": ([ctypes.POINTER(Config), ctypes.POINTER(vp)], ci),
            "es_sur_destroy": ([vp], None),
            "es_sur_set_stream": ([vp, vp], ci),
            "es_sur_num_params": ([vp], ctypes.c_longlong),
            "es_sur_get_params": ([vp, vp], ci),
            "es_sur_set_params": ([vp, vp], ci),
            "es_sur_set_output_scale": ([vp, ctypes.POINTER(cf)], ci),
            "es_sur_fit_output_scale": ([vp, vp, ci], ci),
            "es_sur_predict": ([vp, vp, vp, ci, vp], ci),
            "es_sur_loss_grad": ([vp, vp, vp, vp, ci, ctypes.POINTER(cf), vp, vp], ci),
            "es_sur_train_step": ([vp, vp, vp, vp, ci, cf, ctypes.POINTER(cf)], ci),
            "es_gemm_bf16": ([ci, ci, ci, vp, ci, ci, vp, ci, ci, vp, ci, cf, cf, ci, vp], ci),
            "es_gemm_status": ([], ci),
            "es_gemm_wait_probe": ([ctypes.c_double, vp], ci),
            "es_sur_combine": ([vp, ci, ctypes.c_longlong, vp, vp, ci, vp, vp], ci),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _bound = True
    return lib


def _dp(t):
    import torch
    if not (t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(rc, where):
    if rc != 0:
        raise _es.EsError(rc, where)


def es_gemm_status():
    """Synchronizes the device; raises EsError if a bounded wait of the
    tcgen05 GEMM ran out since the last call (es_gemm_status)."""
    _check(_lib().es_gemm_status(), "es_gemm_status")


def es_gemm_wait_probe(seconds, stream=None):
    """Runs the bounded-wait failure path on the device (es_gemm_wait_probe):
    one wait on a barrier nothing completes gives up after `seconds`; the next
    es_gemm_status() raises EsError(ES_ERR_TIMEOUT)."""
    _check(_lib().es_gemm_wait_probe(float(seconds), _es._stream_handle(stream)), "es_gemm_wait_probe")


def es_gemm_bf16(A, B, C, a_t=False, b_nk=False, alpha=1.0, beta=0.0, split_k=1, stream=None):
    """C = alpha op(A) op(B) + beta C with torch bf16 A, B and float32 C (CUDA)."""
    M, N = C.shape
    K = A.shape[0] if a_t else A.shape[1]
    lda, ldb = A.shape[1], B.shape[1]
    _check(_lib().es_gemm_bf16(M, N, K, _dp(A), lda, int(a_t), _dp(B), ldb, int(b_nk), _dp(C), N, float(alpha),
                               float(beta), int(split_k), _es._stream_handle(stream)), "es_gemm_bf16")
    return C


class Surrogate:
    """es_sur: position + moment tensor -> 4C seismograms [4][n_rcv][nt]."""

    def __init__(self, n_rcv, nt, nfreq=3, hidden=256, latent=128, max_batch=256, seed=0, stream=None):
        self.lib = _lib()
        self.cfg = Config(nfreq, hidden, latent, n_rcv, nt, max_batch, seed)
        self.D = 4 * n_rcv * nt
        self.max_batch = max_batch
        h = ctypes.c_void_p()
        _check(self.lib.es_sur_create(ctypes.byref(self.cfg), ctypes.byref(h)), "es_sur_create")
        self._h = h
        if stream is not None:
            _check(self.lib.es_sur_set_stream(h, _es._stream_handle(stream)), "es_sur_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            self.lib.es_sur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(self.lib.es_sur_num_params(self._h))

    def get_params(self):
        out = np.empty(self.num_params(), np.float32)
        _check(self.lib.es_sur_get_params(self._h, ctypes.c_void_p(out.ctypes.data)), "es_sur_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        _check(self.lib.es_sur_set_params(self._h, ctypes.c_void_p(p.ctypes.data)), "es_sur_set_params")

    def set_output_scale(self, scale4):
        s = (ctypes.c_float * 4)(*[float(v) for v in scale4])
        _check(self.lib.es_sur_set_output_scale(self._h, s), "es_sur_set_output_scale")

    def fit_output_scale(self, targets):
        _check(self.lib.es_sur_fit_output_scale(self._h, _dp(targets), targets.shape[0]), "es_sur_fit_output_scale")

    def predict(self, pos, mt, out=None):
        import torch
        B = pos.shape[0]
        if out is None:
            out = torch.empty((B, self.D), device=pos.device)
        _check(self.lib.es_sur_predict(self._h, _dp(pos), _dp(mt), B, _dp(out)), "es_sur_predict")
        return out

    def loss_grad(self, pos, mt, target, grads=True):
        import torch
        B = pos.shape[0]
        per = torch.empty(B, device=pos.device)
        g = torch.empty(self.num_params(), device=pos.device) if grads else None
        loss = ctypes.c_float()
        _check(self.lib.es_sur_loss_grad(self._h, _dp(pos), _dp(mt), _dp(target), B, ctypes.byref(loss), _dp(per),
                                         _dp(g) if grads else None), "es_sur_loss_grad")
        return loss.value, per, g

    def train_step(self, pos, mt, target, lr, want_loss=True):
        """One Adam step; returns the batch loss, or None with want_loss=False
        (no device synchronisation: the step stays queued on the stream)."""
        loss = ctypes.c_float()
        _check(self.lib.es_sur_train_step(self._h, _dp(pos), _dp(mt), _dp(target), pos.shape[0], float(lr),
                                          ctypes.byref(loss) if want_loss else None), "es_sur_train_step")
        return loss.value if want_loss else None


# ---------------------------------------------------------------------------
# workflow
# ---------------------------------------------------------------------------

UNIT_MT = np.eye(6)


def normalize_positions(pos, box):
    """Grid cells of the catalog box mapped to [-1, 1]^3 (input side, a rescaling of integers)."""
    lo = np.array([b[0] for b in box], np.float64)
    hi = np.array([b[1] for b in box], np.float64)
    return (2.0 * (np.asarray(pos, np.float64) - lo) / np.maximum(hi - lo, 1.0) - 1.0).astype(np.float32)


def green_catalog(model, locations, nt, dt, rcv, wavelet, per_batch=16):
    """Unit-moment-tensor responses of every catalog location from the solver:
    returns a CUDA tensor G [n_loc][6][4][n_rcv][nt] (component c = Mxx Myy
    Mzz Mxy Mxz Myz set to 1).  model: an es.Model (its sources and batch are
    replaced)."""
    import torch
    n_loc = len(locations)
    n_rcv = len(rcv)
    G = torch.empty((n_loc, 6, 4, n_rcv, nt), device="cuda")
    rcv_d = torch.from_numpy(np.ascontiguousarray(rcv, np.int32)).cuda()
    for s in range(0, n_loc, per_batch):
        locs = locations[s:s + per_batch]
        pos = np.repeat(np.asarray(locs, np.int32), 6, axis=0)
        mts = np.tile(UNIT_MT, (len(locs), 1))
        wav = np.tile(np.asarray(wavelet, np.float32), (len(pos), 1))
        model.batch_set(pos, mts, wav)
        out = G[s:s + len(locs)].view(len(pos), 4, n_rcv, nt)
        model.run(nt, dt, rcv_d, out)
    model.batch_set(pos[:1], mts[:1], wav[:1])
    return G


def combine(G, loc, mt, stream=None):
    """Reference traces of (location, moment tensor) pairs as the exact linear
    combination sum_c M_c G[loc][c] (es_sur_combine).  Returns
    [B][4][n_rcv][nt]."""
    import torch
    n_loc, six, four, n_rcv, nt = G.shape
    B = len(loc)
    out = torch.empty((B, 4, n_rcv, nt), device="cuda")
    if B == 0:
        return out
    li = torch.from_numpy(np.ascontiguousarray(loc, np.int32)).cuda()
    mm = torch.from_numpy(np.ascontiguousarray(mt, np.float32)).cuda()
    _check(_lib().es_sur_combine(_dp(G), n_loc, 4 * n_rcv * nt, _dp(li), _dp(mm), B, _dp(out),
                                 _es._stream_handle(stream)), "es_sur_combine")
    return out


def random_moment_tensors(rng, n):
    """Training draws: half random double couples, half general tensors
    (isotropic and CLVD parts included), each of unit norm."""
    u = rng.uniform(n)
    dc = synth.random_dc_batch(rng, n)
    gen = rng.normal(6 * n).reshape(n, 6)
    out = np.where((u < 0.5)[:, None], dc, gen)
    return out / np.sqrt(np.sum(out[:, :3] ** 2, axis=1) + 2 * np.sum(out[:, 3:] ** 2, axis=1))[:, None]


def train(sur, pos_n, G, epochs, lr=2e-3, batch=None, per_loc=8, seed=0, log=None, warmup=0.02):
    """Adam on the catalog: every epoch draws per_loc fresh moment tensors per
    location (random_moment_tensors) and regresses the network onto their exact
    seismograms (combine).  pos_n: [n_loc][3] normalized positions.  Learning
    rate: linear warm-up over the first `warmup` fraction of the steps, then a
    cosine decay.  Returns the loss of each epoch's last batch."""
    import torch
    n_loc = G.shape[0]
    sur.fit_output_scale(G.view(n_loc * 6, -1))
    batch = batch or sur.max_batch
    rng = synth.SplitMix64(1000 + seed)
    order_rng = np.random.default_rng(seed)
    N = n_loc * per_loc
    n_steps = epochs * max(1, math.ceil(N / batch))
    history, step = [], 0
    pos_dev = torch.from_numpy(np.ascontiguousarray(pos_n, np.float32)).cuda()
    for ep in range(epochs):
        loc = np.repeat(np.arange(n_loc), per_loc)
        mts = random_moment_tensors(rng, N)
        order = order_rng.permutation(N)
        if len(order) % batch:
            order = np.concatenate([order, order[:batch - len(order) % batch]])
        loss = None
        for s in range(0, len(order), batch):
            idx = order[s:s + batch]
            tgt = combine(G, loc[idx], mts[idx]).view(len(idx), -1)
            li = torch.from_numpy(loc[idx]).cuda()
            mm = torch.from_numpy(mts[idx].astype(np.float32)).cuda()
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / n_steps))
            if step < warmup * n_steps:
                lr_t *= (step + 1) / (warmup * n_steps)
            last = s + batch >= len(order)
            # the loss is read back (a synchronisation) once per epoch, on its last batch
            loss = sur.train_step(pos_dev[li].contiguous(), mm, tgt, max(lr_t, 1e-6), want_loss=last)
            step += 1
        history.append(float(loss))
        if log and (ep % max(1, epochs // 10) == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {history[-1]:.3e}")
    return history


def rel_errors(sur, pos_n, loc, mt, truth, batch=None):
    """Per source, the relative L2 error of the surrogate's 4C seismogram
    against `truth` [B][4][n_rcv][nt], each component divided by the
    network's output scale for it (pressure and velocity differ by orders of
    magnitude)."""
    import torch
    batch = batch or sur.max_batch
    B = len(loc)
    errs = np.empty(B)
    for s in range(0, B, batch):
        n = min(batch, B - s)
        m = (n + 7) // 8 * 8
        idx = list(range(s, s + n)) + [s] * (m - n)
        p = torch.from_numpy(pos_n[np.asarray(loc)[idx]]).cuda()
        mm = torch.from_numpy(np.asarray(mt, np.float32)[idx]).cuda()
        t = truth[idx].reshape(m, -1).contiguous()
        _, per, _ = sur.loss_grad(p, mm, t, grads=False)
        errs[s:s + n] = np.sqrt(per.cpu().numpy()[:n])
    return errs


def calibrate_gate(sur, pos_n, G, n_val=4, threshold=0.05, margin=0.8, seed=7):
    """Error gate: for every catalog location, n_val held-out random double
    couples are predicted and compared with their exact solver-built
    references; a location is trusted when all its errors stay below
    margin * threshold.  Returns (trusted [n_loc] bool, errors [n_loc][n_val])."""
    n_loc = G.shape[0]
    rng = synth.SplitMix64(seed)
    loc = np.repeat(np.arange(n_loc), n_val)
    mts = np.array([synth.random_dc(rng) for _ in range(len(loc))])
    truth = combine(G, loc, mts)
    errs = rel_errors(sur, pos_n, loc, mts, truth).reshape(n_loc, n_val)
    return errs.max(axis=1) <= margin * threshold, errs


def serve(sur, pos_n, trusted, loc, mt, solver_model, locations, nt, dt, rcv, wavelet, batch_solver=16, out=None):
    """Seismograms for sources (location index, moment tensor): the surrogate
    where the gate trusts the location, the solver (batched runs) elsewhere.
    out: optional contiguous CUDA float32 [B][4][n_rcv][nt] to fill (a reused
    serving buffer).  Returns (traces CUDA [B][4][n_rcv][nt], used_solver bool
    [B])."""
    import torch
    B = len(loc)
    n_rcv = len(rcv)
    if out is None:
        out = torch.empty((B, 4, n_rcv, nt), device="cuda")
    elif tuple(out.shape) != (B, 4, n_rcv, nt) or not out.is_contiguous() or out.dtype != torch.float32:
        raise ValueError("serve: out must be a contiguous float32 [B][4][n_rcv][nt] CUDA tensor")
    flat = out.view(B, -1)
    use_sur = trusted[np.asarray(loc)]
    idx = np.nonzero(use_sur)[0]
    if len(idx):
        # the inputs of every trusted source in one copy each; a run of consecutive sources
        # (all of them when every location is trusted) is predicted straight into the output
        p_all = torch.from_numpy(np.ascontiguousarray(pos_n[np.asarray(loc)[idx]], np.float32)).cuda()
        m_all = torch.from_numpy(np.ascontiguousarray(np.asarray(mt, np.float32)[idx])).cuda()
        run = idx[-1] - idx[0] == len(idx) - 1
        for s in range(0, len(idx), sur.max_batch):
            part = idx[s:s + sur.max_batch]
            n = len(part)
            if run and n % 8 == 0:
                sur.predict(p_all[s:s + n], m_all[s:s + n], out=flat[part[0]:part[0] + n])
                continue
            pad = (n + 7) // 8 * 8 - n
            p = torch.cat([p_all[s:s + n], p_all[s:s + 1].expand(pad, 3)]).contiguous()
            mm = torch.cat([m_all[s:s + n], m_all[s:s + 1].expand(pad, 6)]).contiguous()
            y = sur.predict(p, mm)
            out[torch.from_numpy(part).cuda()] = y[:n].view(n, 4, n_rcv, nt)
    rest = np.nonzero(~use_sur)[0]
    rcv_d = torch.from_numpy(np.ascontiguousarray(rcv, np.int32)).cuda()
    for s in range(0, len(rest), batch_solver):
        part = rest[s:s + batch_solver]
        pos = np.asarray(locations, np.int32)[np.asarray(loc)[part]]
        wav = np.tile(np.asarray(wavelet, np.float32), (len(part), 1))
        solver_model.batch_set(pos, np.asarray(mt)[part], wav)
        tr = torch.empty((len(part), 4, n_rcv, nt), device="cuda")
        solver_model.run(nt, dt, rcv_d, tr)
        out[torch.from_numpy(part).cuda()] = tr
    return out, ~use_sur


# ---------------------------------------------------------------------------
# sources away from the catalog: exact references, baselines, the position
# gate and serving with the solver as the fallback
# ---------------------------------------------------------------------------

def solver_references(model, pos, mt, nt, dt, rcv, wavelet, per_batch=32):
    """Exact 4C seismograms [B][4][n_rcv][nt] (CUDA) of moment-tensor sources at
    arbitrary grid cells, from batched solver runs (one simulation per source).
    model: an es.Model (its sources and batch are replaced)."""
    import torch
    B, n_rcv = len(pos), len(rcv)
    out = torch.empty((B, 4, n_rcv, nt), device="cuda")
    rcv_d = torch.from_numpy(np.ascontiguousarray(rcv, np.int32)).cuda()
    for s in range(0, B, per_batch):
        part = np.arange(s, min(B, s + per_batch))
        wav = np.tile(np.asarray(wavelet, np.float32), (len(part), 1))
        model.batch_set(np.asarray(pos, np.int32)[part], np.asarray(mt)[part], wav)
        model.run(nt, dt, rcv_d, out[s:s + len(part)])
    return out


def nearest_locations(locations, pos, k=1):
    """The k catalog locations nearest to each position (Euclidean distance in
    cells): (indices [B][k], distances [B][k])."""
    loc = np.asarray(locations, np.float64)
    p = np.asarray(pos, np.float64)
    d2 = ((p[:, None, :] - loc[None, :, :]) ** 2).sum(axis=2)
    idx = np.argsort(d2, axis=1, kind="stable")[:, :k]
    return idx, np.sqrt(np.take_along_axis(d2, idx, axis=1))


def baseline_nearest(G, locations, pos, mt):
    """Baseline without a network: the exact seismogram of the same moment
    tensor at the nearest catalog location."""
    idx, _ = nearest_locations(locations, pos, 1)
    return combine(G, idx[:, 0], mt)


def baseline_idw(G, locations, pos, mt, k=8):
    """Baseline without a network: the catalog interpolated to the position by
    inverse-distance-squared weights over its k nearest locations (each term
    the exact seismogram of the weighted moment tensor there; at a catalog
    location, that location alone)."""
    idx, dist = nearest_locations(locations, pos, k)
    w = 1.0 / np.maximum(dist, 1e-9) ** 2
    w = np.where(dist[:, :1] < 1e-9, (dist < 1e-9).astype(np.float64), w)
    w /= w.sum(axis=1, keepdims=True)
    mt = np.asarray(mt, np.float64)
    out = None
    for j in range(k):
        part = combine(G, idx[:, j], w[:, j:j + 1] * mt)
        out = part if out is None else out.add_(part)
    return out


def predict_at(sur, box, pos, mt):
    """The network's seismograms [B][4][n_rcv][nt] for sources at arbitrary
    cells of the box (positions normalised as for training)."""
    import torch
    B = len(pos)
    pn = normalize_positions(pos, box)
    out = torch.empty((B, sur.D), device="cuda")
    for s in range(0, B, sur.max_batch):
        n = min(sur.max_batch, B - s)
        m = (n + 7) // 8 * 8
        idx = np.concatenate([np.arange(s, s + n), np.full(m - n, s)])
        y = sur.predict(torch.from_numpy(pn[idx]).cuda(), torch.from_numpy(np.asarray(mt, np.float32)[idx]).cuda())
        out[s:s + n] = y[:n]
    return out.view(B, 4, -1, sur.cfg.nt)


def component_scale(G):
    """RMS of each of the 4 components over the catalog, shape [1][4][1][1]:
    the weights of the whole-seismogram relative L2 (pressure and velocity
    differ by orders of magnitude)."""
    return G.permute(2, 0, 1, 3, 4).reshape(4, -1).pow(2).mean(dim=1).sqrt().view(1, 4, 1, 1)


def scaled_rel_l2(pred, truth, scale):
    """Per source, the relative L2 of the 4C seismogram with each component
    divided by its scale; numpy [B]."""
    B = truth.shape[0]
    d = ((pred - truth) / scale).reshape(B, -1).norm(dim=1)
    return (d / (truth / scale).reshape(B, -1).norm(dim=1)).cpu().numpy()


def calibrate_position_gate(dist, err, threshold=0.05, margin=0.8):
    """Gate for sources away from the catalog from held-out sources: the
    largest distance d* to the nearest catalog location such that every
    held-out source at a distance up to d* (and above 0) has an error below
    margin * threshold; -1 when the nearest off-catalog held-out source is
    already above it (only catalog locations are served by the network)."""
    dist, err = np.asarray(dist, np.float64), np.asarray(err, np.float64)
    off = dist > 0
    order = np.argsort(dist[off], kind="stable")
    ds, es_ = dist[off][order], err[off][order]
    ok = es_ <= margin * threshold
    if len(ds) == 0 or not ok[0]:
        return -1.0
    first_bad = np.argmin(ok) if not ok.all() else len(ok)
    return float(ds[first_bad - 1])


def serve_positions(sur, box, trusted_loc, d_star, locations, pos, mt, solver_model, nt, dt, rcv, wavelet,
                    batch_solver=32, out=None):
    """Seismograms for sources at arbitrary cells: the network where the source
    sits on a catalog location the location gate trusts, or within d_star cells
    of the catalog; the solver (batched runs at the exact positions) elsewhere.
    Returns (traces CUDA [B][4][n_rcv][nt], used_solver bool [B])."""
    import torch
    B, n_rcv = len(pos), len(rcv)
    if out is None:
        out = torch.empty((B, 4, n_rcv, nt), device="cuda")
    idx, dist = nearest_locations(locations, pos, 1)
    on_cat = dist[:, 0] < 1e-9
    use_sur = np.where(on_cat, np.asarray(trusted_loc)[idx[:, 0]], dist[:, 0] <= d_star)
    net = np.nonzero(use_sur)[0]
    if len(net):
        out[torch.from_numpy(net).cuda()] = predict_at(sur, box, np.asarray(pos)[net], np.asarray(mt)[net])
    rest = np.nonzero(~use_sur)[0]
    if len(rest):
        ref = solver_references(solver_model, np.asarray(pos)[rest], np.asarray(mt)[rest], nt, dt, rcv, wavelet,
                                per_batch=batch_solver)
        out[torch.from_numpy(rest).cuda()] = ref
    return out, ~use_sur
