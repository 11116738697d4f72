"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module generates signals only: it holds none of the transform's
arithmetic and imports nothing else from this package, so both the FP64 oracle
checks and the CUDA path can be fed from it.  Every generator is a pure function
of its seed (NumPy's PCG64, identical on x86 and Arm), returning complex64
arrays in the library's layout (batch-major, transform elements contiguous;
2D frames row-major).

Workload recipes (the paper measures on no public dataset; these stand in for
its radar workloads):

* ``uniform``      -- iid U[-1, 1] real and imaginary parts.
* ``uniform_hash`` -- the same distribution from a counter-based hash
                      (SplitMix64): the host twin of the library's on-device
                      generator ``fft_fill_uniform``, bit for bit.
* ``tones``        -- per transform, unit-amplitude complex exponentials at
                      seeded integer bins; the forward DFT of one tone at bin k0
                      is N at k0 and 0 elsewhere.
* ``buried_tone``  -- ``uniform`` plus a tone of amplitude 1e-3 at a seeded bin
                      in every transform (mixed-precision accuracy workload).
* ``sar_frame``    -- a [azimuth rows][range cols] frame of linear-FM chirp
                      echoes (bandwidth-time product 500, sampled at 1.2x the
                      bandwidth, so 600-sample chirps in both directions) from
                      point scatterers with unit amplitude and uniform random
                      phase, plus circular complex Gaussian noise at the given
                      SNR relative to the mean signal power of the frame.
"""
from __future__ import annotations

import numpy as np

__all__ = ["uniform", "uniform_hash", "tones", "tone_bins", "buried_tone", "sar_frame", "chirp"]


def uniform(seed: int, batch: int, n: int) -> np.ndarray:
    """(batch, n) complex64 with iid U[-1, 1] real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=(batch, n)).astype(np.float32)
    im = rng.uniform(-1.0, 1.0, size=(batch, n)).astype(np.float32)
    out = np.empty((batch, n), dtype=np.complex64)
    out.real = re
    out.imag = im
    return out


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def uniform_hash(seed: int, count: int, first: int = 0) -> np.ndarray:
    """(count,) complex64: values first .. first + count - 1 of the seeded
    counter-based sequence the library's fft_fill_uniform writes on the
    device.  SplitMix64 (Steele, Lea, Flood 2014) at stream index k: state
    seed + (k + 1) * 0x9E3779B97F4A7C15, two xor-shift-multiply rounds and a
    final xor-shift; the top 24 bits u give 2 u 2^-24 - 1 in [-1, 1).  Element
    j takes indices 2 (first + j) (real part) and 2 (first + j) + 1."""
    with np.errstate(over="ignore"):
        k = (np.uint64(2) * (np.uint64(first) + np.arange(count, dtype=np.uint64)))
        k = np.stack([k, k + np.uint64(1)], axis=-1).reshape(-1)
        z = np.uint64(seed & (2 ** 64 - 1)) + (k + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
    v = np.float32(2.0) * u - np.float32(1.0)
    out = np.empty(count, dtype=np.complex64)
    out.real = v[0::2]
    out.imag = v[1::2]
    return out


def tone_bins(seed: int, batch: int, n: int, ntones: int = 1) -> np.ndarray:
    """(batch, ntones) int64 distinct bins in [0, n) used by ``tones``."""
    rng = np.random.default_rng(seed)
    k = min(ntones, n)
    return np.stack([rng.choice(n, size=k, replace=False) for _ in range(batch)])


def _exp_bins(bins: np.ndarray, n: int) -> np.ndarray:
    """exp(+2 pi i k j / n) for j < n, one row per bin k; the phase index k*j is
    reduced mod n as an integer before the angle is formed."""
    j = np.arange(n, dtype=np.int64)
    ph = (bins[:, None].astype(np.int64) * j[None, :]) % n
    ang = 2.0 * np.pi * ph.astype(np.float64) / float(n)
    return np.cos(ang) + 1j * np.sin(ang)


def tones(seed: int, batch: int, n: int, ntones: int = 1) -> np.ndarray:
    """(batch, n) complex64: sum of ``ntones`` unit tones per transform at the
    bins returned by ``tone_bins(seed, batch, n, ntones)``."""
    bins = tone_bins(seed, batch, n, ntones)
    out = np.zeros((batch, n), dtype=np.complex128)
    for b in range(batch):
        out[b] = _exp_bins(bins[b], n).sum(axis=0)
    return out.astype(np.complex64)


def buried_tone(seed: int, batch: int, n: int, amplitude: float = 1e-3):
    """``uniform`` plus one tone of the given amplitude at a seeded bin per
    transform.  Returns (x complex64 (batch, n), bins int64 (batch,))."""
    x = uniform(seed, batch, n)
    bins = np.random.default_rng(seed + 0x5EED).integers(0, n, size=batch)
    # exp(2 pi i m / n) for m < n, indexed by the integer-reduced phase k*j mod n:
    # the same values _exp_bins forms, computed once
    table = _exp_bins(np.ones(1, dtype=np.int64), n)[0]
    j = np.arange(n, dtype=np.int64)
    rows = max(1, (1 << 22) // max(n, 1))          # rows per chunk: bounded host memory
    for b0 in range(0, batch, rows):
        b1 = min(batch, b0 + rows)
        tone = table[(bins[b0:b1, None].astype(np.int64) * j[None, :]) % n]
        x[b0:b1] = (x[b0:b1].astype(np.complex128) + amplitude * tone).astype(np.complex64)
    return x, bins


def chirp(bt: float = 500.0, oversample: float = 1.2) -> np.ndarray:
    """Baseband linear-FM chirp sampled at ``oversample`` x its bandwidth:
    L = round(oversample * bt) samples, phase pi * (j - L/2)^2 / (oversample^2 bt)."""
    length = int(round(oversample * bt))
    t = np.arange(length, dtype=np.float64) - length / 2.0
    return np.exp(1j * np.pi * t * t / (oversample * oversample * bt))


def sar_frame(seed: int, rows: int = 4096, cols: int = 8192, scatterers: int = 50,
              bt: float = 500.0, snr_db: float = 10.0, oversample: float = 1.2) -> np.ndarray:
    """(rows, cols) complex64 SAR raw-data frame: azimuth along rows, range
    along the contiguous columns."""
    rng = np.random.default_rng(seed)
    c = chirp(bt, oversample)
    length = c.size
    frame = np.zeros((rows, cols), dtype=np.complex128)
    r0 = rng.integers(0, rows, size=scatterers)
    c0 = rng.integers(0, cols, size=scatterers)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=scatterers)
    half = length // 2
    for s in range(scatterers):
        ra, rb = r0[s] - half, r0[s] - half + length
        ca, cb = c0[s] - half, c0[s] - half + length
        ia, ib = max(ra, 0), min(rb, rows)
        ja, jb = max(ca, 0), min(cb, cols)
        if ia >= ib or ja >= jb:
            continue
        patch = np.exp(1j * phase[s]) * np.outer(c[ia - ra:ib - ra], c[ja - ca:jb - ca])
        frame[ia:ib, ja:jb] += patch
    power = np.mean(np.abs(frame) ** 2)
    sigma2 = power / (10.0 ** (snr_db / 10.0))
    noise = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    frame += np.sqrt(sigma2 / 2.0) * noise
    return frame.astype(np.complex64)


def azimuth_rate(cols: int, col, length: int):
    """Azimuth chirp rate (cycles / sample^2) of range bin ``col``: 0.8 / length
    at near range, falling to 0.8 / (1.5 length) at far range, so the
    azimuth bandwidth stays below the pulse repetition frequency."""
    return 0.8 / length / (1.0 + 0.5 * np.asarray(col, dtype=np.float64) / cols)


def sar_raw(seed: int, rows: int = 4096, cols: int = 8192, scatterers: int = 50,
            bt: float = 500.0, azimuth_len: int = 512, snr_db: float = 10.0,
            oversample: float = 1.2):
    """SAR raw data of point scatterers without range migration, with the
    replicas a range-Doppler processor correlates against.

    Returns ``(frame, range_replica, azimuth_replicas, positions)``:
      frame             (rows, cols) complex64, azimuth along rows, range along
                        the contiguous columns; scatterer s at (r0, c0) adds
                        exp(i phi_s) * a_{c0}(r - r0) * g(c - c0), circularly;
      range_replica     (cols,) complex64: the transmitted chirp g (``chirp``),
                        starting at sample 0, zero-padded;
      azimuth_replicas  (rows, cols) complex64: column c holds that range bin's
                        azimuth chirp a_c(t) = exp(i pi K_c t^2) for
                        t in [-azimuth_len/2, azimuth_len/2), at row t mod rows
                        (K_c from ``azimuth_rate``);
      positions         (scatterers, 2) int64 (r0, c0).
    Complex Gaussian noise is added at ``snr_db`` below the mean signal power."""
    rng = np.random.default_rng(seed)
    g = chirp(bt, oversample)
    lr, la = g.size, int(azimuth_len)
    if lr > cols or la > rows:
        raise ValueError("chirps longer than the frame")
    t = np.arange(la, dtype=np.float64) - la // 2
    r0 = rng.integers(0, rows, size=scatterers)
    c0 = rng.integers(0, cols, size=scatterers)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=scatterers)
    frame = np.zeros((rows, cols), dtype=np.complex128)
    ci_base = np.arange(lr)
    for s in range(scatterers):
        a = np.exp(1j * np.pi * azimuth_rate(cols, c0[s], la) * t * t)
        ri = (r0[s] + t.astype(np.int64)) % rows
        ci = (c0[s] + ci_base) % cols
        frame[np.ix_(ri, ci)] += np.exp(1j * phase[s]) * np.outer(a, g)
    power = np.mean(np.abs(frame) ** 2)
    sigma2 = power / (10.0 ** (snr_db / 10.0))
    noise = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    frame += np.sqrt(sigma2 / 2.0) * noise
    range_replica = np.zeros(cols, dtype=np.complex64)
    range_replica[:lr] = g
    k = azimuth_rate(cols, np.arange(cols), la)
    az = np.zeros((rows, cols), dtype=np.complex64)
    az[t.astype(np.int64) % rows, :] = np.exp(1j * np.pi * np.outer(t * t, k))
    return (frame.astype(np.complex64), range_replica, az,
            np.stack([r0, c0], axis=1).astype(np.int64))
