"""Seeded synthetic inputs shared by the tests, the oracle checks and the
benchmark.  This module holds no arithmetic of the correlation-function
method: it only draws fields.

Lognormal recipe (stands in for the MHD ISM density cubes of Sec. 4, which
are not available here):
  1. white noise w ~ N(0, 1): counter-based splitmix64 draws (two per cell,
     counter 2i and 2i+1 of a seed-derived stream) turned into a normal by
     Box-Muller;
  2. g_hat = FFT(w) * sqrt(P(|k|)), k = 2 pi f / N per axis, P(0) = 0, and an
     optional Gaussian cutoff P <- P exp(-(k/k_c)^2 / 2);
  3. g = IFFT(g_hat) (real), rescaled to zero mean and standard deviation
     sigma_G;
  4. delta = exp(g - sigma_G^2 / 2) - 1, minus its sample mean;
  5. cast to the requested dtype.
Particle recipe (the validation input of Sec. 4.3): `n` distinct random cells
set to weight 1 on an otherwise empty grid.
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """splitmix64 output function applied to a uint64 array of counters."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniforms(seed, n, stream=0):
    """n uniforms in (0, 1) from counters seed-stream-mixed with 0..n-1."""
    base = splitmix64(np.array([np.uint64(seed) * np.uint64(1000003) + np.uint64(stream)],
                               dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        ctr = (np.arange(n, dtype=np.uint64) + base) & _M64
    z = splitmix64(ctr)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def white_noise(seed, shape):
    n = int(np.prod(shape))
    u = uniforms(seed, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)


def gaussian_field(seed, shape, slope, cutoff=None):
    """Gaussian random field with P(k) ~ k^slope (zero mean, unit variance)."""
    w = white_noise(seed, shape)
    ks = [2.0 * np.pi * np.fft.fftfreq(n) for n in shape[:-1]]
    ks.append(2.0 * np.pi * np.fft.rfftfreq(shape[-1]))
    grids = np.meshgrid(*ks, indexing="ij", sparse=True)
    k = np.sqrt(sum(g * g for g in grids))
    with np.errstate(divide="ignore"):
        p = np.where(k > 0, k ** float(slope), 0.0)
    if cutoff is not None:
        p = p * np.exp(-0.5 * (k / cutoff) ** 2)
    g = np.fft.irfftn(np.fft.rfftn(w) * np.sqrt(p), s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    return g / g.std()


def lognormal_field(seed, shape, sigma_g, slope, cutoff=None, dtype=np.float32):
    g = sigma_g * gaussian_field(seed, shape, slope, cutoff)
    d = np.exp(g - 0.5 * sigma_g * sigma_g) - 1.0
    d -= d.mean()
    return d.astype(dtype)


def particle_field(seed, shape, n, dtype=np.float64):
    """n distinct cells of weight 1 (Sec. 4.3 validation input)."""
    total = int(np.prod(shape))
    u = uniforms(seed, 8 * n + 64, stream=7)
    picks, seen = [], set()
    for v in u:
        c = int(v * total)
        if c not in seen:
            seen.add(c)
            picks.append(c)
            if len(picks) == n:
                break
    f = np.zeros(total, dtype=dtype)
    f[picks] = 1.0
    return f.reshape(shape)


# Workloads named by what they are (the configurations of the benchmark).
def edges_linear(lo, hi, nbins):
    return np.linspace(lo, hi, nbins + 1)


def edges_log(lo, hi, nbins):
    return np.geomspace(lo, hi, nbins + 1)


WORKLOADS = {
    # projected 3PCF, 64^2 float64, sigma_G 1.0, P ~ k^-2, edges {2,5,8,11,14}, mmax 4
    "proj64_3pcf": dict(shape=(64, 64), dtype=np.float64, sigma=1.0, slope=-2.0, cutoff=None,
                        edges=[2.0, 5.0, 8.0, 11.0, 14.0], seed=1001),
    # full 128^3 float32, sigma 1.2, P ~ k^-3 with Gaussian cutoff at k_Nyq/2, 8 linear bins 2..18
    "full128": dict(shape=(128, 128, 128), dtype=np.float32, sigma=1.2, slope=-3.0,
                    cutoff=np.pi / 2, edges=list(edges_linear(2.0, 18.0, 8)), seed=1002),
    # full 256^3 float32, sigma 1.5, P ~ k^-11/3, 10 linear bins 2..32
    "full256": dict(shape=(256, 256, 256), dtype=np.float32, sigma=1.5, slope=-11.0 / 3.0,
                    cutoff=None, edges=list(edges_linear(2.0, 32.0, 10)), seed=1003),
    # full 512^3 float32, sigma 1.5, P ~ k^-11/3, 20 linear bins 2..62
    "full512": dict(shape=(512, 512, 512), dtype=np.float32, sigma=1.5, slope=-11.0 / 3.0,
                    cutoff=None, edges=list(edges_linear(2.0, 62.0, 20)), seed=1005),
}


def workload_field(name):
    w = WORKLOADS[name]
    return lognormal_field(w["seed"], w["shape"], w["sigma"], w["slope"], w["cutoff"], w["dtype"])


def batch_member(j):
    """Field j of the 64-field projected batch: sizes 128^2..1024^2 (16 each),
    sigma_G in [0.5, 2] from the seed, P ~ k^-8/3, 10 log bins 2..N/8."""
    n = (128, 256, 512, 1024)[j // 16]
    seed = 4000 + j
    sigma = 0.5 + 1.5 * float(uniforms(seed, 1, stream=3)[0])
    f = lognormal_field(seed, (n, n), sigma, -8.0 / 3.0, None, np.float32)
    return f, list(edges_log(2.0, n / 8.0, 10))
