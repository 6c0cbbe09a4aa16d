"""Seeded synthetic inputs shaped like the paper's workloads.

The paper refactors Gray-Scott reaction-diffusion output (Sec. IV.A), which is
not available here; it notes that the refactoring time does not depend on the
values, so seeded synthetic fields of the same shapes stand in for it.  This
module only generates inputs (fields and coordinates); it contains none of the
decomposition's arithmetic and serves both the CUDA path and the CPU oracle.

Workloads (by name)
  sines65       65^3 FP64, unit spacing: sum of three seeded sines with random
                wave vectors |k| <= 4 cycles per domain plus N(0, 1e-3) noise.
  grf513        513^3 (2^9+1, Sec. IV.B's kernel size): Gaussian random field
                with power spectrum |k|^-5/3 synthesised by FFT, normalised to
                mean 0 / variance 1.
  bumps_stretched_1000x700x300
                1000 x 700 x 300 (not 2^k+1), geometric coordinates
                h_i = 1.01^i per axis: smooth low-frequency product of cosines
                plus 32 Gaussian bumps (centres uniform in index space, widths
                2..20 cells, N(0,1) amplitudes).
  batch_field_specs: 4096 uneven 2D / 3D fields for the batched form.
"""
import numpy as np

try:
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)


def uniform_coords(shape):
    return [np.arange(n, dtype=np.float64) for n in shape]


def stretched_coords(n, ratio=1.01, h0=1.0):
    """x_0 = 0, x_{i+1} - x_i = h0 * ratio**i (formed in FP64)."""
    return np.concatenate([[0.0], np.cumsum(h0 * ratio ** np.arange(n - 1, dtype=np.float64))])


def sines_field(shape, seed=0, n_waves=3, kmax=4.0, noise=1e-3):
    """Sum of seeded sines, wave vectors uniform in the ball |k| <= kmax."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) / (n - 1) for n in shape], indexing="ij")
    u = np.zeros(shape)
    for _ in range(n_waves):
        while True:
            k = rng.uniform(-kmax, kmax, d)
            if np.linalg.norm(k) <= kmax:
                break
        phi = rng.uniform(0, 2 * np.pi)
        u += np.sin(2 * np.pi * sum(k[i] * grids[i] for i in range(d)) + phi)
    u += rng.normal(0.0, noise, shape)
    return u


def grf_field(shape, seed=0, slope=-5.0 / 3.0):
    """Gaussian random field with power |k|^slope (amplitude |k|^(slope/2))."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    spec = _rfftn(white)
    del white
    d = len(shape)
    k2 = None
    for ax in range(d):
        n = shape[ax]
        if ax == d - 1:
            k = np.fft.rfftfreq(n) * n
        else:
            k = np.fft.fftfreq(n) * n
        sh = [1] * d
        sh[ax] = k.shape[0]
        term = (k.reshape(sh)) ** 2
        k2 = term if k2 is None else k2 + term
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)
    spec *= amp
    del amp, k2
    u = _irfftn(spec, s=shape)
    del spec
    u -= u.mean()
    u /= u.std()
    return u


def bumps_field(shape, seed=0, n_bumps=32, coords=None):
    """Smooth product of cosines over normalised coordinates plus Gaussian bumps."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    if coords is None:
        coords = [stretched_coords(n) for n in shape]
    xn = [(c - c[0]) / (c[-1] - c[0]) for c in coords]
    freqs = rng.uniform(0.5, 2.0, d)
    phases = rng.uniform(0, 2 * np.pi, d)
    smooth = [np.cos(2 * np.pi * freqs[k] * xn[k] + phases[k]) for k in range(d)]
    centres = [rng.uniform(0, shape[k] - 1, n_bumps) for k in range(d)]
    widths = rng.uniform(2.0, 20.0, n_bumps)
    amps = rng.standard_normal(n_bumps)
    idx = [np.arange(n, dtype=np.float64) for n in shape]
    # separable factors: g[k][b, i] = exp(-((i - c_b)/sigma_b)^2 / 2)
    g = [np.exp(-0.5 * ((idx[k][None, :] - centres[k][:, None]) / widths[:, None]) ** 2) for k in range(d)]
    out = np.empty(shape, dtype=np.float64)
    if d == 1:
        out[:] = smooth[0] + (amps[:, None] * g[0]).sum(0)
        return out
    rest_shape = shape[1:]
    # rest[b, ...] = outer product of the factors of axes 1..d-1 for bump b
    rest = g[1]
    for k in range(2, d):
        rest = (rest[:, :, None] * g[k][:, None, :]).reshape(n_bumps, -1)
    rest = rest.reshape(n_bumps, -1)
    smooth_rest = smooth[1]
    for k in range(2, d):
        smooth_rest = np.multiply.outer(smooth_rest, smooth[k])
    smooth_rest = smooth_rest.reshape(-1)
    lead = (amps[:, None] * g[0]).T  # (n0, n_bumps)
    chunk = max(1, int(2 ** 26 // max(1, rest.shape[1])))
    flat = out.reshape(shape[0], -1)
    for i0 in range(0, shape[0], chunk):
        i1 = min(shape[0], i0 + chunk)
        flat[i0:i1] = lead[i0:i1] @ rest
        flat[i0:i1] += smooth[0][i0:i1, None] * smooth_rest[None, :]
    return out


WORKLOADS = {
    "sines65": dict(shape=(65, 65, 65), dtype="f64", coords="uniform"),
    "grf513": dict(shape=(513, 513, 513), dtype="f64", coords="uniform"),
    "bumps_stretched_1000x700x300": dict(shape=(1000, 700, 300), dtype="f32", coords="stretched"),
}


def workload(name, seed=0, shape=None):
    """(field, coords) of a named workload; coords is None for unit spacing."""
    spec = WORKLOADS[name]
    shape = tuple(shape) if shape is not None else spec["shape"]
    if name == "sines65":
        return sines_field(shape, seed), None
    if name == "grf513":
        return grf_field(shape, seed), None
    coords = [stretched_coords(n) for n in shape]
    return bumps_field(shape, seed, coords=coords), coords


# ---------------------------------------------------------------------------
# thousands of uneven fields for the batched form
# ---------------------------------------------------------------------------

def batch_field_specs(count=4096, seed=0):
    """(shape, stretched) of the batched workload.

    Element count N is log-uniform on [17^2, 129^3]; N <= 129^2 gives a
    near-square 2D field, larger N a near-cube 3D field; every side is in
    [17, 129] and not forced to 2^k+1; half the fields (p = 1/2) use
    geometric coordinates with ratio 1.01 per cell, the others unit spacing.
    """
    rng = np.random.default_rng(seed)
    lo, hi = np.log(17.0 ** 2), np.log(129.0 ** 3)
    specs = []
    for _ in range(count):
        n = float(np.exp(rng.uniform(lo, hi)))
        if n <= 129.0 ** 2:
            a = int(np.clip(round(np.sqrt(n) * rng.uniform(0.85, 1.15)), 17, 129))
            b = int(np.clip(round(n / a), 17, 129))
            shape = (a, b)
        else:
            a = int(np.clip(round(n ** (1.0 / 3.0) * rng.uniform(0.85, 1.15)), 17, 129))
            b = int(np.clip(round((n / a) ** 0.5 * rng.uniform(0.9, 1.1)), 17, 129))
            c = int(np.clip(round(n / (a * b)), 17, 129))
            shape = (a, b, c)
        specs.append((shape, bool(rng.random() < 0.5)))
    return specs


def grf_field_torch(shape, seed=0, slope=-5.0 / 3.0, device="cuda"):
    """Gaussian random field with power |k|^slope, generated with torch on
    `device` from a seeded generator (same recipe as grf_field); FP64 result,
    mean 0 and variance 1."""
    import torch

    g = torch.Generator(device=device).manual_seed(int(seed))
    white = torch.randn(tuple(shape), generator=g, device=device, dtype=torch.float64)
    spec = torch.fft.rfftn(white)
    d = len(shape)
    k2 = None
    for ax in range(d):
        n = shape[ax]
        k = (torch.fft.rfftfreq(n, device=device) if ax == d - 1 else torch.fft.fftfreq(n, device=device)) * n
        sh = [1] * d
        sh[ax] = k.shape[0]
        term = k.reshape(sh).to(torch.float64) ** 2
        k2 = term if k2 is None else k2 + term
    amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (slope / 4.0), torch.zeros_like(k2))
    u = torch.fft.irfftn(spec * amp, s=tuple(shape))
    u = u - u.mean()
    return u / u.std()
