"""Helpers for the GPU parity tests: run the CUDA path through the C ABI with
torch-owned device buffers and return numpy arrays."""
import numpy as np
import torch

from paper_0903_3852_gb300 import build as sde_build
from paper_0903_3852_gb300 import sde

_built = False


def ensure_built():
    global _built
    if not _built:
        sde_build.build()
        assert torch.cuda.is_available(), "GPU tests need a CUDA device"
        _built = True
    return sde.lib()


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def jj_run(ens, x0, v0, n_begin, n_end, w0=None, vs0=None):
    """Advance a Josephson ensemble on the GPU; returns (x_abs, v, w, x_frac, vsum, obs)."""
    x_in, v_in = dev(x0, torch.float32), dev(v0, torch.float32)
    w_in = None if w0 is None else dev(w0, torch.int32)
    vs_in = None if vs0 is None else dev(vs0, torch.float64)
    n = x_in.numel()
    x_out = torch.empty(n, dtype=torch.float32, device="cuda")
    v_out = torch.empty_like(x_out)
    w_out = torch.empty(n, dtype=torch.int32, device="cuda")
    vs_out = torch.empty(n, dtype=torch.float64, device="cuda")
    ens.run_josephson(n_begin, n_end, x_in, v_in, x_out, v_out, w_out, vs_out, w_in=w_in, vsum_in=vs_in)
    obs = ens.observables()
    x = x_out.cpu().numpy()
    w = w_out.cpu().numpy()
    return (w.astype(np.float64) + x.astype(np.float64), v_out.cpu().numpy().astype(np.float64), w, x,
            vs_out.cpu().numpy(), obs)


def mixed_rel(a, ref):
    return np.abs(np.asarray(a, np.float64) - ref) / np.maximum(1.0, np.abs(ref))


def kur_run(ens, phi0, omega, n_begin, n_end):
    phi_in = dev(phi0, torch.float32)
    om = dev(omega, torch.float32)
    phi_out = torch.empty_like(phi_in)
    M = ens.sample_every
    rows = (-(-(n_end - n_begin) // M) + 1) if M > 0 else 0
    r_out = torch.zeros((max(rows, 1), ens.n_replicas), dtype=torch.float64, device="cuda")
    ens.run_kuramoto(n_begin, n_end, phi_in, phi_out, om, r_out=r_out if rows else None)
    obs = ens.observables()
    return phi_out.cpu().numpy().astype(np.float64), r_out.cpu().numpy()[:rows], obs


def angle_diff(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return (d + np.pi) % (2 * np.pi) - np.pi
