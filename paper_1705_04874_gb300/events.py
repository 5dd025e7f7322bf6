"""Clustered microseismic events (Sec. VI-A of Das, Chen & Hobson, arXiv
1705.04874): event locations are kept where the Laplacian of the density
(Eq. (8)) exceeds a threshold -- rock interfaces, where faults are likely --
the kept events are grouped into clusters whose origin times lie close
together, and es_superpose turns their single-event traces into one record.

The Laplacian runs on the GPU (es_laplacian: the solver's own spectral
derivative passes); the selection and the draws are host bookkeeping.  The
grouping into clusters (the paper compares k-means, Gaussian mixtures and
hierarchical clustering) is the caller's: pass the labels in."""
from __future__ import annotations

import numpy as np

from . import es, synth


def density_laplacian(rho, d=(10.0, 10.0, 10.0)):
    """Spectral Laplacian of the density [nz][ny][nx] (numpy or CUDA tensor)
    with spacings d = (dx, dy, dz): a CUDA tensor of the same shape."""
    import torch
    f = rho if torch.is_tensor(rho) else torch.from_numpy(np.ascontiguousarray(rho, np.float32))
    f = f.cuda().contiguous()
    out = torch.empty_like(f)
    es.es_laplacian(f, d, out)
    return out


def select_event_locations(lap, locations, threshold=0.1):
    """Indices into `locations` ([n][3] cells (ix, iy, iz)) whose |Laplacian|
    exceeds `threshold` (the paper keeps |L| > 0.1), and the Laplacian values
    there (FP32, the decision is taken in FP32)."""
    import torch
    loc = np.asarray(locations, np.int64)
    idx = torch.from_numpy(loc[:, 2] * lap.shape[1] * lap.shape[2] + loc[:, 1] * lap.shape[2] + loc[:, 0])
    vals = lap.reshape(-1)[idx.to(lap.device)].cpu().numpy()
    return np.nonzero(np.abs(vals) > np.float32(threshold))[0], vals


def clustered_events(rng: synth.SplitMix64, labels, amp_sigma=1.0, between=0.3, within_sd=0.1):
    """One event per selected location (src_of_event = 0 .. n-1 in the order of
    `labels`): log-normal amplitudes (sigma amp_sigma, Sec. IV-C) and origin
    times grouped by cluster (synth.cluster_origin_times: cluster c starts at
    c * between seconds, events spread by N(0, within_sd)).  Returns
    (src_of_event int32, amps float32, t0s float32) for es_superpose."""
    labels = np.asarray(labels)
    n = labels.size
    amps = np.exp(amp_sigma * rng.normal(n)).astype(np.float32)
    t0s = synth.cluster_origin_times(rng, labels, between=between, within_sd=within_sd)
    return np.arange(n, dtype=np.int32), amps, t0s
