"""Seeded synthetic fusion problems (host-only NumPy, float64).

Generates the inputs that both the CUDA path and the FP64 oracle consume:
ground truth Z, the guide/high-resolution image Y_h = Z R + N_h, the
low-resolution image Y_l = S(b * Z) + N_l, the blur kernel b, the spectral
response R and the subspace basis E.  This module holds none of the solver's
arithmetic: it only synthesises data following the imaging model of Sec. I-A
(eq. model) and the subspace representation Z = X E (Sec. I-A).  The blur used
for synthesis is an FFT-based circular convolution written here for data
generation only.

Layout of every image returned: planar band-major float64 arrays of shape
(L, H, W) (band c is image[c]); this is the layout of the C-ABI.

Spatial structure (stand-in for the paper's Pleiades/Pavia/Chikusei/CAVE
scenes, which are not available): periodic smooth Gaussian random fields plus
tiled periodic texture patches over random rectangles, which gives the
repeated (self-similar) structure that a nonlocal patch prior targets.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 2210041840


@dataclasses.dataclass
class Problem:
    """One synthetic fusion problem (all arrays float64, images planar (L, H, W))."""
    H: int
    W: int
    L_l: int
    L_h: int
    L_s: int
    d: int
    K: int
    S: int
    lam1: float
    lam2: float
    rho: float
    h: float
    iters: int
    blur: np.ndarray      # (bh, bw), centred, sums to 1
    R: np.ndarray         # (L_l, L_h)
    E: np.ndarray         # (L_s, L_l)
    Z: np.ndarray         # (L_l, H, W) ground truth
    Yh: np.ndarray        # (L_h, H, W)
    Yl: np.ndarray        # (L_l, H/d, W/d)
    name: str = ""

    @property
    def guide(self) -> np.ndarray:
        return self.Yh


def gaussian_kernel(size: int, sigma: float) -> np.ndarray:
    r = size // 2
    u = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def _rescale01(a: np.ndarray) -> np.ndarray:
    lo, hi = a.min(), a.max()
    return (a - lo) / (hi - lo) if hi > lo else np.zeros_like(a)


def smooth_field(rng, H: int, W: int, corr: float) -> np.ndarray:
    """Periodic smooth Gaussian random field with correlation length `corr` px, in [0, 1]."""
    noise = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    spec = np.exp(-2.0 * (np.pi * corr) ** 2 * (fy ** 2 + fx ** 2))
    f = np.fft.ifft2(np.fft.fft2(noise) * spec).real
    return _rescale01(f)


def textured_field(rng, H: int, W: int, corr: float, tile: int = 16, nrect: int = 6) -> np.ndarray:
    """Smooth field with a random periodic tile pasted over random rectangles, in [0, 1]."""
    base = smooth_field(rng, H, W, corr)
    t = rng.random((tile, tile))
    tiled = np.tile(t, (-(-H // tile), -(-W // tile)))[:H, :W]
    mask = np.zeros((H, W))
    for _ in range(nrect):
        h0 = int(rng.integers(0, H)); w0 = int(rng.integers(0, W))
        hh = int(rng.integers(max(2, H // 8), max(3, H // 3)))
        ww = int(rng.integers(max(2, W // 8), max(3, W // 3)))
        rows = (np.arange(h0, h0 + hh) % H)[:, None]
        cols = (np.arange(w0, w0 + ww) % W)[None, :]
        mask[rows, cols] = 1.0
    return _rescale01((1.0 - mask) * base + mask * (0.35 * base + 0.65 * tiled))


def endmember_spectra(rng, n_end: int, L: int) -> np.ndarray:
    """Smooth random curves over band index: sums of 3 Gaussians, clipped at 0. (n_end, L)."""
    b = np.arange(L, dtype=np.float64)
    out = np.zeros((n_end, L))
    for e in range(n_end):
        for _ in range(3):
            c = rng.uniform(0, L); w = rng.uniform(L / 12, L / 3); a = rng.uniform(0.2, 1.0)
            out[e] += a * np.exp(-0.5 * ((b - c) / w) ** 2)
    return np.clip(out, 0.0, None)


def band_gaussian_response(L: int, n_out: int) -> np.ndarray:
    """Band-localised Gaussian responses, centres evenly spaced, width L/8; columns sum to 1."""
    b = np.arange(L, dtype=np.float64)[:, None]
    centres = (np.arange(n_out) + 0.5) * L / n_out
    R = np.exp(-0.5 * ((b - centres[None, :]) / (L / 8.0)) ** 2)
    return R / R.sum(axis=0, keepdims=True)


def _circ_blur_fft(Z: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """Data synthesis only: circular convolution of every band with a centred kernel."""
    L, H, W = Z.shape
    bh, bw = kern.shape
    img = np.zeros((H, W))
    for a in range(bh):
        for c in range(bw):
            img[(a - bh // 2) % H, (c - bw // 2) % W] += kern[a, c]
    kf = np.fft.fft2(img)
    return np.fft.ifft2(np.fft.fft2(Z, axes=(1, 2)) * kf[None], axes=(1, 2)).real


def _add_noise(rng, Y: np.ndarray, snr_db: float) -> np.ndarray:
    """Per band, i.i.d. Gaussian with variance mean(Y_c^2) / 10^(SNR/10)."""
    if snr_db is None or not np.isfinite(snr_db):
        return Y.copy()
    p = (Y ** 2).reshape(Y.shape[0], -1).mean(axis=1)
    sig = np.sqrt(p / 10.0 ** (snr_db / 10.0))
    return Y + sig[:, None, None] * rng.standard_normal(Y.shape)


def subspace_basis(Yl: np.ndarray, L_s: int) -> np.ndarray:
    """Top-L_s right singular vectors of Y_l (n_l x L_l), rows orthonormal, sign fixed. (L_s, L_l)."""
    L = Yl.shape[0]
    if L_s == L:
        return np.eye(L)
    M = Yl.reshape(L, -1).T
    _, _, vt = np.linalg.svd(M, full_matrices=False)
    E = vt[:L_s].copy()
    for r in range(L_s):
        j = int(np.argmax(np.abs(E[r])))
        if E[r, j] < 0:
            E[r] = -E[r]
    return E


def make_problem(*, H, W, L_l, L_h, L_s, d=4, blur_size=9, blur_sigma=1.7, snr_l=35.0,
                 snr_h=35.0, K=1, S=2, lam1=1.0, lam2=1e-3, rho=1e-2, h=0.15, iters=50,
                 seed=0, kind="hsms", n_end=6, E_identity=False, name="") -> Problem:
    """Build one seeded problem. kind: 'pansharpen' (random fields, random nonnegative R),
    'hsms' (endmember mixtures, band-localised R), 'hspan' (endmember mixtures, ramp R)."""
    rng = np.random.default_rng(seed)
    corr = max(H, W) / 16.0
    if kind == "pansharpen":
        Z = np.stack([textured_field(rng, H, W, corr) for _ in range(L_l)])
        R = rng.random((L_l, L_h))
        R /= R.sum(axis=0, keepdims=True)
    else:
        spectra = endmember_spectra(rng, n_end, L_l)
        logits = np.stack([4.0 * textured_field(rng, H, W, corr) for _ in range(n_end)])
        ab = np.exp(logits - logits.max(axis=0, keepdims=True))
        ab /= ab.sum(axis=0, keepdims=True)
        Z = np.einsum("ehw,el->lhw", ab, spectra)
        Z = _rescale01(Z)
        if kind == "hspan":
            r = 1.0 + np.arange(L_l) / float(L_l)
            R = (r / r.sum())[:, None] * np.ones((1, L_h))
        else:
            R = band_gaussian_response(L_l, L_h)
    blur = gaussian_kernel(blur_size, blur_sigma)
    Yh = _add_noise(rng, np.einsum("lhw,lk->khw", Z, R), snr_h)
    Yl = _add_noise(rng, _circ_blur_fft(Z, blur)[:, ::d, ::d], snr_l)
    E = np.eye(L_l) if E_identity else subspace_basis(Yl, L_s)
    if E_identity:
        L_s = L_l
    return Problem(H=H, W=W, L_l=L_l, L_h=L_h, L_s=L_s, d=d, K=K, S=S, lam1=lam1, lam2=lam2,
                   rho=rho, h=h, iters=iters, blur=blur, R=R, E=E, Z=Z, Yh=Yh,
                   Yl=np.ascontiguousarray(Yl), name=name)


# The workloads (sizes, bands, blur, noise, patch/search windows, iterations).
# lambda1 = 1 and h = 0.15 for every workload; lambda2 = 1e-3, rho = 1e-2.
WORKLOADS = {
    # Pansharpening MS+PAN, FP64: Z 128x128x4, PAN 1 band, 9x9 sigma 1.7, d 4, 40 dB,
    # patch 3x3 (K=1), search 5x5 (S=2, 24 offsets), 50 iterations.
    "pansharpen_128": dict(H=128, W=128, L_l=4, L_h=1, L_s=4, d=4, blur_size=9, blur_sigma=1.7,
                           snr_l=40.0, snr_h=40.0, K=1, S=2, iters=50, kind="pansharpen",
                           E_identity=True, dtype="f64", wdtype="f64", cfg=0),
    # HS+MS fusion, FP32 with BF16 weights: Z 256x256x93, MS 4 bands, HS 64x64x93,
    # 9x9 sigma 1.7, 35 dB, patch 5x5 (K=2), search 7x7 (S=3, 48 offsets), 100 iterations,
    # subspace L_s = 20.
    "hsms_256": dict(H=256, W=256, L_l=93, L_h=4, L_s=20, d=4, blur_size=9, blur_sigma=1.7,
                     snr_l=35.0, snr_h=35.0, K=2, S=3, iters=100, kind="hsms",
                     dtype="f32", wdtype="bf16", cfg=1),
    # HS+PAN sharpening, FP32: Z 512x512x128, PAN 1 band (flat-plus-ramp R), 11x11 sigma 2,
    # 30 dB, patch 5x5, search 11x11 (S=5, 120 offsets), 200 iterations, L_s = 20.
    "hspan_512": dict(H=512, W=512, L_l=128, L_h=1, L_s=20, d=4, blur_size=11, blur_sigma=2.0,
                      snr_l=30.0, snr_h=30.0, K=2, S=5, iters=200, kind="hspan",
                      dtype="f32", wdtype="bf16", cfg=2),
    # The HS+MS workload at 128 x 128 (same bands, windows and iterations): latent state 1.6 GB,
    # above L2 but small enough for detailed profiler captures.
    "hsms_128": dict(H=128, W=128, L_l=93, L_h=4, L_s=20, d=4, blur_size=9, blur_sigma=1.7,
                     snr_l=35.0, snr_h=35.0, K=2, S=3, iters=100, kind="hsms",
                     dtype="f32", wdtype="bf16", cfg=1),
    # Unrolled forward of the differentiable form: Z 256x256x31, MS 3 bands, sigma 1.5,
    # patch 3x3, search 3x3 (S=1), 20 iterations, L_s = 8.
    "unrolled_256": dict(H=256, W=256, L_l=31, L_h=3, L_s=8, d=4, blur_size=9, blur_sigma=1.5,
                         snr_l=35.0, snr_h=35.0, K=1, S=1, iters=20, kind="hsms",
                         dtype="f32", wdtype="f32", cfg=3),
    # Guided inpainting (a variant of the same ADMM): Z 256x256x31, 20% of the pixels observed at
    # random (S a random mask, no blur), an MS guide of 3 bands, patch 3x3, search 7x7, 100
    # iterations, L_s = 8, BF16 weights.
    "inpaint_256": dict(H=256, W=256, L_l=31, L_h=3, L_s=8, d=1, blur_size=1, blur_sigma=1.0,
                        snr_l=35.0, snr_h=35.0, K=1, S=3, iters=100, kind="hsms",
                        dtype="f32", wdtype="bf16", cfg=5, mask_fraction=0.2),
}


def sampling_mask(H: int, W: int, fraction: float, seed: int) -> np.ndarray:
    """A seeded random 0/1 mask (uint8, H x W) keeping about `fraction` of the pixels."""
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) < fraction).astype(np.uint8)


def workload(name: str, **override) -> tuple[Problem, dict]:
    """Build a named workload; returns (problem, meta) with meta holding dtype/wdtype."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    dtype = spec.pop("dtype"); wdtype = spec.pop("wdtype"); cfg = spec.pop("cfg")
    seed = spec.pop("seed", SEED_BASE + cfg)
    frac = spec.pop("mask_fraction", None)
    p = make_problem(seed=seed, name=name, **spec)
    meta = dict(dtype=dtype, wdtype=wdtype, seed=seed)
    if frac is not None:
        meta["mask"] = sampling_mask(p.H, p.W, frac, seed + 1)
    return p, meta


def batch_sizes(n: int = 64, seed: int = SEED_BASE + 4) -> list[int]:
    """Square sizes for the batched uneven-tile workload, uniform over {96,...,384}."""
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.choice([96, 128, 192, 256, 320, 384], size=n)]


def batch_workload(n: int = 64, seed: int = SEED_BASE + 4, sizes=None) -> list[Problem]:
    """The batched uneven-tile workload: n HS+MS problems, square sizes uniform over
    {96, 128, 192, 256, 320, 384}, 31 bands, MS 3 bands, ratio 4, 9x9 blur (sigma 1.7), 35 dB,
    patch 3x3 (K=1), search 7x7 (S=3), L_s = 8, 100 iterations each."""
    sizes = sizes if sizes is not None else batch_sizes(n, seed)
    return [make_problem(H=sz, W=sz, L_l=31, L_h=3, L_s=8, d=4, blur_size=9, blur_sigma=1.7, snr_l=35.0,
                         snr_h=35.0, K=1, S=3, iters=100, kind="hsms", seed=seed + 1000 * (i + 1),
                         name=f"batch{i}_{sz}")
            for i, sz in enumerate(sizes)]
