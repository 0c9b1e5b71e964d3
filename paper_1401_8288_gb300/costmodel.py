"""The paper's sizing equations, and the work counts the benchmark reports.

Host-side arithmetic only.  Eq. 1-4 are the paper's (Sec. 2.2.3 and Sec. 2.4);
``cmacs`` is the X-stage work in complex multiply-accumulates that the
benchmark's MACs/s figure is based on.
"""

from __future__ import annotations

import math


def n_pairs(n_inputs: int) -> int:
    """Input pairs of the lower triangle, autos included: N_i (N_i + 1) / 2.
    Eq. 1 counts 8 flops for each of them per sample (4 N_i (N_i + 1))."""
    return n_inputs * (n_inputs + 1) // 2


def gpu_flops(n_inputs: int, bandwidth_hz: float) -> float:
    """Eq. 1: R = 4 N_i (N_i + 1) N_c / tau, in single-precision flop/s.

    N_c / tau is the processed bandwidth (N_c channels, each sampled at the
    Nyquist interval tau of the F-engine spectra)."""
    return 4.0 * n_inputs * (n_inputs + 1) * bandwidth_hz


def input_bits_per_s(n_inputs: int, bandwidth_hz: float) -> float:
    """Eq. 2: D = 8 N_i N_c / tau bit/s (4 + 4 bits per complex sample)."""
    return 8.0 * n_inputs * bandwidth_hz


def server_capture_bits_per_s(n_fpga: int, inputs_per_fpga: int, ch_low: int,
                              ch_high: int, n_servers: int, tau_s: float) -> float:
    """Eq. 3: D_I = 8 N_r N_a (High_ch - Low_ch) / (N_serv tau)."""
    return 8.0 * n_fpga * inputs_per_fpga * (ch_high - ch_low) / (n_servers * tau_s)


def output_size_eq4(n_chan: int, n_inputs: int, n_pol: int = 2) -> float:
    """Eq. 4 as printed: D_cc = N_c (N_i / 4 + 1)(N_i / 2) N_pol^2.

    The library stores the exact packed triangle (``n_pairs``) instead; this
    helper only reproduces the paper's count."""
    return n_chan * (n_inputs / 4 + 1) * (n_inputs / 2) * n_pol ** 2


def gpus_needed(flops_required: float, flops_per_gpu: float) -> int:
    """Table 1's GPU counts: the smallest whole number of GPUs whose combined
    rate strictly exceeds the requirement (every printed count, e.g. 105 / 3
    -> 36 and 144324 / 3 -> 48109, follows this reading)."""
    return math.floor(flops_required / flops_per_gpu) + 1


def cmacs(n_chan: int, n_time: int, n_inputs: int) -> int:
    """Complex multiply-accumulates of one X-stage pass: C * K * P."""
    return n_chan * n_time * n_pairs(n_inputs)


def int8_ops(n_chan: int, n_time: int, n_inputs: int) -> int:
    """Integer tensor operations of the same pass: each complex MAC is four
    real multiply-adds, two operations each."""
    return 8 * cmacs(n_chan, n_time, n_inputs)
