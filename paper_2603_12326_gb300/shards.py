"""Loss-table binning of q points spread over several ranks.

Every q of the path is independent up to the rate integral, which needs the
loss functions of all q binned over |q+G| (the momentum grid of the q
integral; end of Appendix A with Eq. (excitation_rate)).  Ranks holding
disjoint sets of q bin their own tables (qcx_bin_loss); the bin means of the
union follow from each rank's bin sums and counts, which one all-reduce (sum)
over the process group combines.  The rank that runs the FP64 rate then
evaluates it on the combined table.  This is the one data exchange of the
multi-GPU path.
"""
from __future__ import annotations

import numpy as np


def combine_bins(mean: np.ndarray, count: np.ndarray, device=None):
    """Global (mean [nbin][nw], count [nbin]) of the q sets of every rank
    from this rank's bin means and counts (host arrays; empty bins are 0).
    `device` is where the collective runs (a CUDA device for NCCL, None or
    "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    nbin, nw = mean.shape
    flat = np.concatenate([(mean * count[:, None]).reshape(-1), count]).astype(np.float64)
    buf = torch.from_numpy(flat)
    if device is not None:
        buf = buf.to(device)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    tot = buf.cpu().numpy()
    sums, cnt = tot[:nbin * nw].reshape(nbin, nw), tot[nbin * nw:]
    out = np.zeros_like(sums)
    nz = cnt > 0
    out[nz] = sums[nz] / cnt[nz][:, None]
    return out, cnt
