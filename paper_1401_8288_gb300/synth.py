"""Seeded synthetic inputs for the X-stage, in the F-stage's output formats.

These generators stand in for the channelised antenna data of the paper's field
system (Sec. 4: 4-bit real + 4-bit imaginary spectra per channel, requantised
on the FPGA, Sec. 2.3 and Fig. 2), which is not available here.  They produce
the sample arrays only; they hold none of the correlation arithmetic, and the
test-suite feeds the same arrays to the oracle and to the CUDA library.

Formats (sample order is always [time][channel][station][pol]):

* CI4  -- one byte per complex sample: the high nibble is the real part and
  the low nibble the imaginary part, each a 4-bit two's-complement integer in
  [-8, 7].  The paper fixes "4 bits real and 4 bits imaginary" (Sec. 2.3,
  Sec. 4) but not the nibble order or the encoding; this is the reading used
  throughout the library.
* CI8  -- two int8 per complex sample, (re, im) interleaved.
* CF32 -- two float32 per complex sample, (re, im) interleaved.

Every generator is deterministic for a given seed: numpy ``Generator(PCG64)``,
filled in fixed-size blocks of time samples so that the stream does not depend
on the caller.
"""

from __future__ import annotations

import numpy as np

_BLOCK_T = 64  # time samples drawn per block; part of the stream definition


def pack_ci4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer real/imaginary parts in [-8, 7] into CI4 bytes."""
    re = np.asarray(re)
    im = np.asarray(im)
    if re.size and (re.min() < -8 or re.max() > 7 or im.min() < -8 or im.max() > 7):
        raise ValueError("CI4 components must lie in [-8, 7]")
    hi = (re.astype(np.int16) & 0xF).astype(np.uint8)
    lo = (im.astype(np.int16) & 0xF).astype(np.uint8)
    return (hi << 4) | lo


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_ci4(n_time: int, n_chan: int, n_sta: int, seed: int,
                lo: int = -7, hi: int = 7) -> np.ndarray:
    """i.i.d. uniform integer components in [lo, hi], packed CI4.

    Shape ``uint8[n_time][n_chan][n_sta][2]``.
    """
    rng = _rng(seed)
    out = np.empty((n_time, n_chan, n_sta, 2), dtype=np.uint8)
    for t0 in range(0, n_time, _BLOCK_T):
        t1 = min(n_time, t0 + _BLOCK_T)
        shape = (t1 - t0, n_chan, n_sta, 2)
        re = rng.integers(lo, hi + 1, size=shape, dtype=np.int8)
        im = rng.integers(lo, hi + 1, size=shape, dtype=np.int8)
        out[t0:t1] = pack_ci4(re, im)
    return out


def _delay_phases(rng: np.random.Generator, n_chan: int, n_sta: int) -> np.ndarray:
    """Per-station geometric phase per channel: a random delay (in samples of the
    channelised band, uniform in [-4, 4)) plus a random constant offset."""
    delay = rng.uniform(-4.0, 4.0, size=n_sta)
    offset = rng.uniform(0.0, 2.0 * np.pi, size=n_sta)
    freq = (np.arange(n_chan) + 0.5) / n_chan
    return 2.0 * np.pi * freq[:, None] * delay[None, :] + offset[None, :]  # [chan][sta]


def gaussian_planewave_ci4(n_time: int, n_chan: int, n_sta: int, seed: int,
                           sigma: float = 2.5, amp: float = 0.3) -> np.ndarray:
    """Gaussian noise plus one common noise-like plane-wave source, CI4.

    Each component of the receiver noise is N(0, sigma^2).  The source is a
    complex signal s[t, c] with N(0, 1) components, scaled by ``amp * sigma``
    and given the phase of station s's delay in channel c (same for both
    polarisations).  The sum is rounded to the nearest integer (half to even)
    and clipped to [-7, 7].  Shape ``uint8[n_time][n_chan][n_sta][2]``.
    """
    rng = _rng(seed)
    phase = _delay_phases(rng, n_chan, n_sta)
    rot = np.exp(1j * phase).astype(np.complex64)  # [chan][sta]
    out = np.empty((n_time, n_chan, n_sta, 2), dtype=np.uint8)
    a = np.float32(amp * sigma)
    for t0 in range(0, n_time, _BLOCK_T):
        t1 = min(n_time, t0 + _BLOCK_T)
        nt = t1 - t0
        noise = rng.standard_normal(size=(nt, n_chan, n_sta, 2, 2), dtype=np.float32)
        noise *= np.float32(sigma)
        src = rng.standard_normal(size=(nt, n_chan, 2), dtype=np.float32)
        s = (src[..., 0] + 1j * src[..., 1]).astype(np.complex64)  # [t][chan]
        v = (a * s[:, :, None] * rot[None, :, :])  # [t][chan][sta]
        re = noise[..., 0] + v.real[..., None]
        im = noise[..., 1] + v.imag[..., None]
        re = np.clip(np.rint(re), -7, 7).astype(np.int8)
        im = np.clip(np.rint(im), -7, 7).astype(np.int8)
        out[t0:t1] = pack_ci4(re, im)
    return out


def gaussian_ci8(n_time: int, n_chan: int, n_sta: int, seed: int,
                 sigma: float = 20.0, clip: int = 127) -> np.ndarray:
    """Complex int8 samples, components N(0, sigma^2) rounded and clipped to
    [-clip, clip].  Shape ``int8[n_time][n_chan][n_sta][2][2]`` (last axis re, im)."""
    rng = _rng(seed)
    out = np.empty((n_time, n_chan, n_sta, 2, 2), dtype=np.int8)
    for t0 in range(0, n_time, _BLOCK_T):
        t1 = min(n_time, t0 + _BLOCK_T)
        g = rng.standard_normal(size=(t1 - t0, n_chan, n_sta, 2, 2), dtype=np.float32)
        g *= np.float32(sigma)
        out[t0:t1] = np.clip(np.rint(g), -clip, clip).astype(np.int8)
    return out


def uniform_ci8(n_time: int, n_chan: int, n_sta: int, seed: int,
                lo: int = -128, hi: int = 127) -> np.ndarray:
    """i.i.d. uniform int8 components in [lo, hi] (the full code range by
    default, -128 included).  Shape ``int8[n_time][n_chan][n_sta][2][2]``."""
    rng = _rng(seed)
    out = np.empty((n_time, n_chan, n_sta, 2, 2), dtype=np.int8)
    for t0 in range(0, n_time, _BLOCK_T):
        t1 = min(n_time, t0 + _BLOCK_T)
        out[t0:t1] = rng.integers(lo, hi + 1, size=(t1 - t0, n_chan, n_sta, 2, 2),
                                  dtype=np.int8)
    return out


def gaussian_cf32(n_time: int, n_chan: int, n_sta: int, seed: int,
                  sigma: float = 1.0) -> np.ndarray:
    """Complex float32 spectra with N(0, sigma^2) components, as a GPU F-stage
    would produce.  Shape ``float32[n_time][n_chan][n_sta][2][2]``."""
    rng = _rng(seed)
    out = np.empty((n_time, n_chan, n_sta, 2, 2), dtype=np.float32)
    for t0 in range(0, n_time, _BLOCK_T):
        t1 = min(n_time, t0 + _BLOCK_T)
        g = rng.standard_normal(size=(t1 - t0, n_chan, n_sta, 2, 2), dtype=np.float32)
        out[t0:t1] = g * np.float32(sigma)
    return out


def quarter_turn_tone_ci4(n_time: int, n_chan: int, n_sta: int, seed: int,
                          amp: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """A noiseless tone whose phase at every input is a whole quarter turn.

    Input i = 2*station + pol in channel c carries ``amp * j**q[c, i]`` at every
    time sample, with q drawn uniformly from {0, 1, 2, 3}; |amp| <= 7 keeps
    every component inside the CI4 range.  Returns ``(packed, q)`` with
    ``q`` of shape ``[n_chan][2*n_sta]``.
    """
    if not 1 <= amp <= 7:
        raise ValueError("amp must be in [1, 7]")
    rng = _rng(seed)
    q = rng.integers(0, 4, size=(n_chan, 2 * n_sta), dtype=np.int8)
    # j**q for q = 0, 1, 2, 3 is 1, j, -1, -j.
    re_of_q = np.array([1, 0, -1, 0], dtype=np.int8)
    im_of_q = np.array([0, 1, 0, -1], dtype=np.int8)
    re = (amp * re_of_q[q]).reshape(n_chan, n_sta, 2)
    im = (amp * im_of_q[q]).reshape(n_chan, n_sta, 2)
    packed = pack_ci4(re, im)
    return np.broadcast_to(packed, (n_time, n_chan, n_sta, 2)).copy(), q


def subarray_batch(seed: int, count: int = 24, inputs=(16, 704), channels=(64, 1024),
                   samples=(512, 8192)) -> list[dict]:
    """Sizes of a batch of independent correlations of uneven size.

    Input counts uniform over the multiples of 16 in ``inputs`` (default
    {16, 32, ..., 704}), channel counts over the multiples of the lower bound
    in ``channels`` (default {64, 128, ..., 1024}), integration lengths over
    the multiples of the lower bound in ``samples`` (default {512, ..., 8192});
    the input count is even (two polarisations per station).  Each entry also
    carries its own sample seed.
    """
    rng = _rng(seed)
    ni = rng.integers(inputs[0] // 16, inputs[1] // 16 + 1, size=count) * 16
    nc = rng.integers(1, channels[1] // channels[0] + 1, size=count) * channels[0]
    nt = rng.integers(1, samples[1] // samples[0] + 1, size=count) * samples[0]
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [dict(n_inputs=int(a), n_sta=int(a) // 2, n_chan=int(b), n_time=int(c),
                 seed=int(s)) for a, b, c, s in zip(ni, nc, nt, seeds)]


def planewave_phases(n_chan: int, n_sta: int, seed: int) -> np.ndarray:
    """The per-station phases [chan][sta] that ``gaussian_planewave_ci4`` gives
    its common source for the same seed (they are its first draws)."""
    return _delay_phases(_rng(seed), n_chan, n_sta)


def uniform_ci4_torch(n_time: int, n_chan: int, n_sta: int, seed: int, device: str = "cuda",
                      lo: int = -7, hi: int = 7):
    """Like ``uniform_ci4`` but drawn on the device with torch's Philox
    generator (a different stream from the numpy one, same distribution):
    for large timing inputs.  Returns a uint8 tensor [n_time][n_chan][n_sta][2]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = (n_time, n_chan, n_sta, 2)
    re = torch.randint(lo, hi + 1, shape, generator=g, device=device, dtype=torch.int16)
    im = torch.randint(lo, hi + 1, shape, generator=g, device=device, dtype=torch.int16)
    return (((re & 0xF) << 4) | (im & 0xF)).to(torch.uint8)


def gaussian_ci4_torch(n_time: int, n_chan: int, n_sta: int, seed: int, sigma: float = 2.5,
                       device: str = "cuda"):
    """Complex Gaussian noise, sigma levels per component, rounded and clipped
    to [-7, 7], drawn on the device (torch Philox): the requantised channel
    data of an F-engine for large streaming inputs.  uint8 [t][c][s][2]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = (n_time, n_chan, n_sta, 2)
    out = torch.empty(shape, dtype=torch.uint8, device=device)
    step = max(1, (1 << 28) // (n_chan * n_sta * 2))  # bounded temporaries
    for t0 in range(0, n_time, step):
        t1 = min(n_time, t0 + step)
        sub = (t1 - t0, n_chan, n_sta, 2)
        re = torch.randn(sub, generator=g, device=device).mul_(sigma).round_().clamp_(-7, 7).to(torch.int16)
        im = torch.randn(sub, generator=g, device=device).mul_(sigma).round_().clamp_(-7, 7).to(torch.int16)
        out[t0:t1] = (((re & 0xF) << 4) | (im & 0xF)).to(torch.uint8)
    return out
