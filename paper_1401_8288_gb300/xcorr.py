"""Thin Python binding of the C ABI in ``include/xcorr.h``.

The functions below carry the C names and only marshal arguments: every step
of the X-stage runs in the library's CUDA kernels.  Device buffers are plain
pointers (``tensor.data_ptr()``) and streams are ``cudaStream_t`` handles
(``torch.cuda.current_stream().cuda_stream``); ``Plan`` wraps both with
PyTorch tensors for convenience.  If the library has not been built this
module raises on first use -- there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

XCORR_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "OVERFLOW",
                5: "CUDA", 6: "DEVICE", 7: "BUDGET"}
XCORR_IN_CI4, XCORR_IN_CI8, XCORR_IN_CF32 = 0, 1, 2
XCORR_ENGINE_AUTO, XCORR_ENGINE_TENSOR, XCORR_ENGINE_CUDA_CORE = 0, 1, 2
XCORR_DUMP_RESET, XCORR_DUMP_ADD_WIDE = 1, 2

FORMATS = {"ci4": XCORR_IN_CI4, "ci8": XCORR_IN_CI8, "cf32": XCORR_IN_CF32}
ENGINES = {"auto": XCORR_ENGINE_AUTO, "tensor": XCORR_ENGINE_TENSOR,
           "cuda_core": XCORR_ENGINE_CUDA_CORE}

EXPORTS = ("xcorr_plan_create", "xcorr_execute", "xcorr_dump", "xcorr_sync", "xcorr_plan_query",
           "xcorr_destroy", "xcorr_last_error", "xcorr_baseline_index", "xcorr_profile_enable",
           "xcorr_profile_read", "xcorr_measure_peak", "xcorr_correlate_ci4_noalloc",
           "xcorr_execute_dump", "xcorr_plan_set_tuning", "xcorr_autotune", "xcorr_batch_create",
           "xcorr_batch_set_variant", "xcorr_batch_execute", "xcorr_batch_capture",
           "xcorr_batch_replay", "xcorr_batch_sync", "xcorr_batch_destroy", "xcorr_tracker_create",
           "xcorr_tracker_feed", "xcorr_tracker_finish", "xcorr_tracker_counters",
           "xcorr_tracker_destroy", "xcorr_packetize", "xcorr_stream_create", "xcorr_stream_acquire",
           "xcorr_stream_commit", "xcorr_stream_flush", "xcorr_stream_counters",
           "xcorr_stream_wait_dump", "xcorr_stream_destroy", "xcorr_packets_advance",
           "xcorr_execute_dump_host", "xcorr_bdi_create", "xcorr_bdi_step", "xcorr_bdi_destroy",
           "xcorr_watchdog_selftest", "xcorr_autotune_cached", "xcorr_tuning_cache_load",
           "xcorr_tuning_cache_save", "xcorr_tuning_cache_clear", "xcorr_batch_set_subarray_variants",
           "xcorr_batch_get_subarray_variants", "xcorr_batch_autotune", "xcorr_accum_load")
XCORR_PACKET_HEADER_BYTES = 16
XCORR_EVENT_OPEN, XCORR_EVENT_CLOSE = 1, 2
PEAK_KINDS = {"tc_e4m3": 0, "tc_bf16": 1, "mma_sync_s8": 2, "dp4a": 3}


class XcorrError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"xcorr {STATUS_NAMES.get(status, status)}: {message}")


class xcorr_config(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int), ("n_pols", ctypes.c_int),
                ("n_channels", ctypes.c_int), ("max_time_per_exec", ctypes.c_int),
                ("fmt", ctypes.c_int), ("engine", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t)]


class xcorr_tuning(ctypes.Structure):
    _fields_ = [("stage_variant", ctypes.c_int), ("groups", ctypes.c_int),
                ("x_streams", ctypes.c_int), ("unfused", ctypes.c_int)]


class xcorr_plan_info(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_channels", ctypes.c_int),
                ("n_pairs", ctypes.c_int64), ("engine", ctypes.c_int),
                ("samples_integrated", ctypes.c_int64), ("max_integration", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("output_bytes", ctypes.c_size_t),
                ("kernels_per_execute", ctypes.c_int), ("tuning", xcorr_tuning)]


class xcorr_stream_config(ctypes.Structure):
    _fields_ = [("n_time_per_packet", ctypes.c_int), ("n_chan_per_packet", ctypes.c_int),
                ("n_inputs_per_packet", ctypes.c_int), ("block_samples", ctypes.c_int),
                ("n_blocks", ctypes.c_int), ("blocks_per_dump", ctypes.c_int),
                ("stack_threshold", ctypes.c_int64), ("chunk_packets", ctypes.c_int64),
                ("n_chunks", ctypes.c_int), ("n_host_dumps", ctypes.c_int)]


class xcorr_packet_counters(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("packets", "placed", "duplicates", "late", "bad", "lost", "blocks_closed")]


class xcorr_block_event(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("slot", ctypes.c_int), ("block", ctypes.c_int64),
                ("position", ctypes.c_int64), ("received", ctypes.c_int64),
                ("lost", ctypes.c_int64)]


class xcorr_dump_record(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("first_seq", ctypes.c_int64), ("n_samples", ctypes.c_int64),
                ("lost_packets", ctypes.c_int64), ("latency_ms", ctypes.c_double),
                ("data", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load ``libxcorr.so`` (build it first with ``paper_1401_8288_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing: build the CUDA library first "
                                   "(python -m paper_1401_8288_gb300.build)")
            lib = ctypes.CDLL(_build.LIB)
            vp, i, u, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_int64
            sig = {
                "xcorr_plan_create": [ctypes.POINTER(vp), ctypes.POINTER(xcorr_config)],
                "xcorr_execute": [vp, vp, i, vp],
                "xcorr_dump": [vp, vp, i, u, vp, ctypes.POINTER(i64)],
                "xcorr_execute_dump": [vp, vp, i, vp, i, u, vp, ctypes.POINTER(i64)],
                "xcorr_accum_load": [vp, vp, i, i64, vp],
                "xcorr_sync": [vp, vp],
                "xcorr_plan_query": [vp, ctypes.POINTER(xcorr_plan_info)],
                "xcorr_destroy": [vp],
                "xcorr_baseline_index": [i, i, i, i, i, ctypes.POINTER(i64), ctypes.POINTER(i)],
                "xcorr_profile_enable": [vp, i],
                "xcorr_profile_read": [vp, ctypes.POINTER(ctypes.c_float), i, ctypes.POINTER(i)],
                "xcorr_measure_peak": [i, ctypes.POINTER(ctypes.c_double)],
                "xcorr_correlate_ci4_noalloc": [vp, i, i, i, vp, vp, vp],
                "xcorr_plan_set_tuning": [vp, ctypes.POINTER(xcorr_tuning)],
                "xcorr_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(xcorr_config), i],
                "xcorr_batch_set_variant": [vp, i],
                "xcorr_batch_execute": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp],
                "xcorr_batch_capture": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp],
                "xcorr_batch_replay": [vp, vp],
                "xcorr_batch_sync": [vp, vp],
                "xcorr_batch_destroy": [vp],
                "xcorr_autotune": [vp, vp, i, vp, ctypes.POINTER(xcorr_tuning),
                                   ctypes.POINTER(ctypes.c_float)],
                "xcorr_autotune_cached": [vp, vp, i, vp, ctypes.POINTER(xcorr_tuning),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i)],
                "xcorr_tuning_cache_load": [ctypes.c_char_p, ctypes.POINTER(i), ctypes.POINTER(i)],
                "xcorr_tuning_cache_save": [ctypes.c_char_p, ctypes.POINTER(i)],
                "xcorr_tuning_cache_clear": [],
                "xcorr_batch_set_subarray_variants": [vp, ctypes.POINTER(i)],
                "xcorr_batch_get_subarray_variants": [vp, ctypes.POINTER(i)],
                "xcorr_batch_autotune": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.POINTER(i)],
                "xcorr_tracker_create": [ctypes.POINTER(vp), ctypes.POINTER(xcorr_stream_config), i,
                                         i],
                "xcorr_tracker_feed": [vp, vp, i64, i64, vp, ctypes.POINTER(xcorr_block_event), i,
                                       ctypes.POINTER(i), ctypes.POINTER(i64)],
                "xcorr_tracker_finish": [vp, ctypes.POINTER(xcorr_block_event), i,
                                         ctypes.POINTER(i)],
                "xcorr_tracker_counters": [vp, ctypes.POINTER(xcorr_packet_counters)],
                "xcorr_tracker_destroy": [vp],
                "xcorr_packetize": [vp, i, i, i, ctypes.POINTER(xcorr_stream_config), i64, vp, i64,
                                    ctypes.POINTER(i64)],
                "xcorr_stream_create": [ctypes.POINTER(vp), vp, ctypes.POINTER(xcorr_stream_config)],
                "xcorr_stream_acquire": [vp, ctypes.POINTER(vp), ctypes.POINTER(i64)],
                "xcorr_stream_commit": [vp, i64],
                "xcorr_stream_flush": [vp],
                "xcorr_stream_counters": [vp, ctypes.POINTER(xcorr_packet_counters),
                                          ctypes.POINTER(i64)],
                "xcorr_stream_wait_dump": [vp, i64, i, ctypes.POINTER(xcorr_dump_record)],
                "xcorr_stream_destroy": [vp],
                "xcorr_packets_advance": [vp, i64, i64, i64],
                "xcorr_execute_dump_host": [vp, vp, i, vp, i, vp],
                "xcorr_bdi_create": [ctypes.POINTER(vp), vp, ctypes.POINTER(i), i],
                "xcorr_bdi_step": [vp, vp, i, vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                   ctypes.POINTER(i64)],
                "xcorr_bdi_destroy": [vp],
                "xcorr_watchdog_selftest": [vp, vp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.xcorr_last_error.argtypes = []
            lib.xcorr_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def xcorr_last_error() -> str:
    return load().xcorr_last_error().decode()


def _check(status: int) -> None:
    if status != XCORR_OK:
        raise XcorrError(status, xcorr_last_error())


def xcorr_plan_create(n_stations: int, n_channels: int, max_time_per_exec: int,
                      fmt: int = XCORR_IN_CI4, engine: int = XCORR_ENGINE_AUTO,
                      hbm_budget_bytes: int = 0, n_pols: int = 2) -> ctypes.c_void_p:
    cfg = xcorr_config(n_stations, n_pols, n_channels, max_time_per_exec, fmt, engine,
                       hbm_budget_bytes)
    plan = ctypes.c_void_p()
    _check(load().xcorr_plan_create(ctypes.byref(plan), ctypes.byref(cfg)))
    return plan


def xcorr_execute(plan, d_in: int, n_time: int, stream: int = 0) -> None:
    _check(load().xcorr_execute(plan, d_in, n_time, stream))


def xcorr_dump(plan, out: int, out_on_device: bool, flags: int = 0, stream: int = 0) -> int:
    n = ctypes.c_int64()
    _check(load().xcorr_dump(plan, out, int(out_on_device), flags, stream, ctypes.byref(n)))
    return n.value


def xcorr_accum_load(plan, src: int, src_on_device: bool, n_samples: int, stream: int = 0) -> None:
    _check(load().xcorr_accum_load(plan, src, int(src_on_device), n_samples, stream))


def xcorr_execute_dump(plan, d_in: int, n_time: int, out: int, out_on_device: bool,
                       flags: int = XCORR_DUMP_RESET, stream: int = 0) -> int:
    n = ctypes.c_int64()
    _check(load().xcorr_execute_dump(plan, d_in, n_time, out, int(out_on_device), flags, stream,
                                     ctypes.byref(n)))
    return n.value


def xcorr_execute_dump_host(plan, h_in: int, n_time: int, h_out: int, n_groups: int = 0,
                            stream: int = 0) -> None:
    _check(load().xcorr_execute_dump_host(plan, h_in, n_time, h_out, n_groups, stream))


def xcorr_watchdog_selftest(plan, stream: int = 0) -> None:
    _check(load().xcorr_watchdog_selftest(plan, stream))


def xcorr_sync(plan, stream: int = 0) -> None:
    _check(load().xcorr_sync(plan, stream))


def _tuning_dict(t: xcorr_tuning) -> dict:
    return {name: getattr(t, name) for name, _ in xcorr_tuning._fields_}


def xcorr_plan_query(plan) -> dict:
    info = xcorr_plan_info()
    _check(load().xcorr_plan_query(plan, ctypes.byref(info)))
    out = {name: getattr(info, name) for name, _ in xcorr_plan_info._fields_}
    out["tuning"] = _tuning_dict(info.tuning)
    return out


def xcorr_plan_set_tuning(plan, stage_variant: int = 0, groups: int = 0, x_streams: int = 2,
                          unfused: int = 0) -> None:
    t = xcorr_tuning(stage_variant, groups, x_streams, unfused)
    _check(load().xcorr_plan_set_tuning(plan, ctypes.byref(t)))


def xcorr_autotune(plan, d_in: int, n_time: int, stream: int = 0) -> tuple[dict, float]:
    """Time every launch shape on this input; the fastest is kept on the plan."""
    t, ms = xcorr_tuning(), ctypes.c_float()
    _check(load().xcorr_autotune(plan, d_in, n_time, stream, ctypes.byref(t), ctypes.byref(ms)))
    return _tuning_dict(t), ms.value


def xcorr_autotune_cached(plan, d_in: int, n_time: int, stream: int = 0) -> tuple[dict, float, bool]:
    """xcorr_autotune through the process's tuning cache: (shape, ms, taken from the cache)."""
    t, ms, hit = xcorr_tuning(), ctypes.c_float(), ctypes.c_int()
    _check(load().xcorr_autotune_cached(plan, d_in, n_time, stream, ctypes.byref(t), ctypes.byref(ms),
                                        ctypes.byref(hit)))
    return _tuning_dict(t), ms.value, bool(hit.value)


def xcorr_tuning_cache_load(path: str) -> tuple[int, int]:
    """Merge a JSON-lines tuning file into the process's cache: (entries loaded, lines skipped)."""
    n, bad = ctypes.c_int(), ctypes.c_int()
    _check(load().xcorr_tuning_cache_load(os.fsencode(path), ctypes.byref(n), ctypes.byref(bad)))
    return n.value, bad.value


def xcorr_tuning_cache_save(path: str) -> int:
    """Write the process's tuning cache to a JSON-lines file; returns the entry count."""
    n = ctypes.c_int()
    _check(load().xcorr_tuning_cache_save(os.fsencode(path), ctypes.byref(n)))
    return n.value


def xcorr_tuning_cache_clear() -> None:
    _check(load().xcorr_tuning_cache_clear())


def xcorr_destroy(plan) -> None:
    _check(load().xcorr_destroy(plan))


def xcorr_baseline_index(n_stations: int, a: int, b: int, p: int, q: int) -> tuple[int, bool]:
    idx, conj = ctypes.c_int64(), ctypes.c_int()
    _check(load().xcorr_baseline_index(n_stations, a, b, p, q, ctypes.byref(idx),
                                       ctypes.byref(conj)))
    return idx.value, bool(conj.value)


def xcorr_profile_enable(plan, capacity: int) -> None:
    _check(load().xcorr_profile_enable(plan, capacity))


def xcorr_profile_read(plan, capacity: int) -> list[tuple[float, float]]:
    """(unpack ms, X-kernel ms) of the last timed executes, oldest first."""
    buf = (ctypes.c_float * (2 * max(capacity, 1)))()
    n = ctypes.c_int()
    _check(load().xcorr_profile_read(plan, buf, capacity, ctypes.byref(n)))
    return [(buf[2 * k], buf[2 * k + 1]) for k in range(n.value)]


def xcorr_measure_peak(kind: str | int) -> float:
    """Measured dense rate (TOPS) of one arithmetic path of the current device."""
    k = PEAK_KINDS.get(kind, kind)
    tops = ctypes.c_double()
    st = load().xcorr_measure_peak(k, ctypes.byref(tops))
    if st != XCORR_OK:
        raise XcorrError(st, f"peak measurement of kind {kind} failed")
    return tops.value


def xcorr_correlate_ci4_noalloc(d_in: int, n_time: int, n_channels: int, n_stations: int,
                                d_out: int, d_status: int = 0, stream: int = 0) -> None:
    """One-shot 4-bit correlation into caller memory, with no device allocation:
    for callers that must not call the allocator (see include/xcorr.h).  Calls
    share one fixed scratch array per GPU, so overlapping calls race."""
    _check(load().xcorr_correlate_ci4_noalloc(d_in, n_time, n_channels, n_stations, d_out,
                                              d_status or None, stream))


def _ptrs(values) -> ctypes.Array:
    return (ctypes.c_void_p * len(values))(*values)


def xcorr_batch_create(subarrays: list[tuple[int, int, int]]) -> ctypes.c_void_p:
    """subarrays: (n_stations, n_channels, n_time) of 4+4-bit correlations."""
    cfgs = (xcorr_config * len(subarrays))(
        *[xcorr_config(ns, 2, nc, nt, XCORR_IN_CI4, XCORR_ENGINE_TENSOR, 0) for ns, nc, nt in subarrays])
    b = ctypes.c_void_p()
    _check(load().xcorr_batch_create(ctypes.byref(b), cfgs, len(subarrays)))
    return b


def xcorr_batch_set_variant(batch, stage_variant: int) -> None:
    _check(load().xcorr_batch_set_variant(batch, stage_variant))


def xcorr_batch_set_subarray_variants(batch, variants: list[int]) -> None:
    _check(load().xcorr_batch_set_subarray_variants(batch, (ctypes.c_int * len(variants))(*variants)))


def xcorr_batch_get_subarray_variants(batch, n: int) -> list[int]:
    v = (ctypes.c_int * n)()
    _check(load().xcorr_batch_get_subarray_variants(batch, v))
    return list(v)


def xcorr_batch_autotune(batch, d_ins: list[int], d_outs: list[int], stream: int = 0) -> list[int]:
    v = (ctypes.c_int * len(d_ins))()
    _check(load().xcorr_batch_autotune(batch, _ptrs(d_ins), _ptrs(d_outs), stream, v))
    return list(v)


def xcorr_batch_execute(batch, d_ins: list[int], d_outs: list[int], stream: int = 0) -> None:
    _check(load().xcorr_batch_execute(batch, _ptrs(d_ins), _ptrs(d_outs), stream))


def xcorr_batch_capture(batch, d_ins: list[int], d_outs: list[int], stream: int = 0) -> None:
    _check(load().xcorr_batch_capture(batch, _ptrs(d_ins), _ptrs(d_outs), stream))


def xcorr_batch_replay(batch, stream: int = 0) -> None:
    _check(load().xcorr_batch_replay(batch, stream))


def xcorr_batch_sync(batch, stream: int = 0) -> None:
    _check(load().xcorr_batch_sync(batch, stream))


def xcorr_batch_destroy(batch) -> None:
    _check(load().xcorr_batch_destroy(batch))


# --------------------------------------------------------------- streaming --
def stream_config(n_time_per_packet: int, n_chan_per_packet: int, n_inputs_per_packet: int,
                  block_samples: int, n_blocks: int = 4, blocks_per_dump: int = 1,
                  stack_threshold: int = 1 << 30, chunk_packets: int = 4096, n_chunks: int = 4,
                  n_host_dumps: int = 2) -> xcorr_stream_config:
    return xcorr_stream_config(n_time_per_packet, n_chan_per_packet, n_inputs_per_packet,
                               block_samples, n_blocks, blocks_per_dump, stack_threshold,
                               chunk_packets, n_chunks, n_host_dumps)


def packet_bytes(cfg: xcorr_stream_config) -> int:
    return (XCORR_PACKET_HEADER_BYTES
            + cfg.n_time_per_packet * cfg.n_chan_per_packet * cfg.n_inputs_per_packet)


def _counters_dict(c: xcorr_packet_counters) -> dict:
    return {name: getattr(c, name) for name, _ in xcorr_packet_counters._fields_}


def xcorr_packetize(samples, cfg: xcorr_stream_config, first_time_block: int = 0):
    """CI4 samples uint8 [t][c][i] (host) -> packets uint8 [n][packet bytes], F-engine order."""
    import numpy as np
    x = np.ascontiguousarray(samples, dtype=np.uint8)
    n_time, n_chan, n_in = x.shape[0], x.shape[1], int(np.prod(x.shape[2:]))
    n_groups, n_feng = n_chan // cfg.n_chan_per_packet, n_in // cfg.n_inputs_per_packet
    cap = (n_time // max(cfg.n_time_per_packet, 1)) * n_groups * n_feng
    out = np.empty((cap, packet_bytes(cfg)), dtype=np.uint8)
    n = ctypes.c_int64()
    _check(load().xcorr_packetize(x.ctypes.data, n_time, n_chan, n_in, ctypes.byref(cfg),
                                  first_time_block, out.ctypes.data, cap, ctypes.byref(n)))
    return out[:n.value]


def xcorr_packets_advance(address: int, stride: int, n: int, seq_delta: int) -> None:
    """Add seq_delta to the sequence numbers of n packets at a host address."""
    _check(load().xcorr_packets_advance(address, stride, n, seq_delta))


class Tracker:
    """Host-side packet tracking (no GPU): placement codes and block events."""

    def __init__(self, cfg: xcorr_stream_config, n_inputs: int, n_channels: int,
                 max_events: int = 1024):
        self.cfg = cfg
        self.handle = ctypes.c_void_p()
        _check(load().xcorr_tracker_create(ctypes.byref(self.handle), ctypes.byref(cfg), n_inputs,
                                           n_channels))
        self._events = (xcorr_block_event * max_events)()
        self._max = max_events

    def _ev_list(self, n: int, offset: int = 0) -> list[dict]:
        return [{"kind": e.kind, "slot": e.slot, "block": e.block, "position": e.position + offset,
                 "received": e.received, "lost": e.lost} for e in self._events[:n]]

    def feed(self, packets):
        """packets: uint8 [n][packet bytes]; returns (codes int64 [n], events)."""
        import numpy as np
        pk = np.ascontiguousarray(packets, dtype=np.uint8)
        n = pk.shape[0]
        codes = np.empty(n, dtype=np.int64)
        events, done = [], 0
        while True:
            n_ev, got = ctypes.c_int(), ctypes.c_int64()
            _check(load().xcorr_tracker_feed(self.handle, pk[done:].ctypes.data if n else None,
                                             pk.shape[1] if pk.ndim == 2 else 16, n - done,
                                             codes[done:].ctypes.data if n else None,
                                             self._events, self._max, ctypes.byref(n_ev),
                                             ctypes.byref(got)))
            events += self._ev_list(n_ev.value, done)
            done += got.value
            if done >= n and n_ev.value < self._max:
                return codes, events

    def finish(self) -> list[dict]:
        events = []
        while True:
            n_ev = ctypes.c_int()
            _check(load().xcorr_tracker_finish(self.handle, self._events, self._max,
                                               ctypes.byref(n_ev)))
            events += self._ev_list(n_ev.value)
            if n_ev.value < self._max:
                return events

    def counters(self) -> dict:
        c = xcorr_packet_counters()
        _check(load().xcorr_tracker_counters(self.handle, ctypes.byref(c)))
        return _counters_dict(c)

    def close(self) -> None:
        if self.handle:
            load().xcorr_tracker_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Stream:
    """A streaming X-stage over a 4-bit plan: push packets, read dumps."""

    def __init__(self, plan: "Plan", cfg: xcorr_stream_config):
        self.plan, self.cfg = plan, cfg
        self.handle = ctypes.c_void_p()
        _check(load().xcorr_stream_create(ctypes.byref(self.handle), plan.handle,
                                          ctypes.byref(cfg)))
        self.packet_bytes = packet_bytes(cfg)
        self.out_shape = (plan.n_channels, plan.info["n_pairs"], 2)

    def acquire(self) -> tuple[int, int]:
        """(host address, capacity in packets) of the next landing chunk."""
        ptr, cap = ctypes.c_void_p(), ctypes.c_int64()
        _check(load().xcorr_stream_acquire(self.handle, ctypes.byref(ptr), ctypes.byref(cap)))
        return ptr.value, cap.value

    def commit(self, n_packets: int) -> None:
        _check(load().xcorr_stream_commit(self.handle, n_packets))

    def push(self, packets) -> None:
        """Copy packets (uint8 [n][packet bytes], host) through the landing chunks."""
        import numpy as np
        pk = np.ascontiguousarray(packets, dtype=np.uint8)
        done = 0
        while done < pk.shape[0]:
            ptr, cap = self.acquire()
            n = min(cap, pk.shape[0] - done)
            ctypes.memmove(ptr, pk[done:done + n].ctypes.data, n * self.packet_bytes)
            self.commit(n)
            done += n

    def flush(self) -> None:
        _check(load().xcorr_stream_flush(self.handle))

    def counters(self) -> tuple[dict, int]:
        c, n = xcorr_packet_counters(), ctypes.c_int64()
        _check(load().xcorr_stream_counters(self.handle, ctypes.byref(c), ctypes.byref(n)))
        return _counters_dict(c), n.value

    def wait_dump(self, k: int, timeout_ms: int = 60000, copy: bool = True) -> dict:
        """Dump k (0-based): its record, with ``data`` an int32 [C][P][2] numpy copy."""
        import numpy as np
        r = xcorr_dump_record()
        _check(load().xcorr_stream_wait_dump(self.handle, k, timeout_ms, ctypes.byref(r)))
        out = {"index": r.index, "first_seq": r.first_seq, "n_samples": r.n_samples,
               "lost_packets": r.lost_packets, "latency_ms": r.latency_ms, "data": None}
        if r.data and copy:
            n = int(np.prod(self.out_shape))
            buf = (ctypes.c_int32 * n).from_address(r.data)
            out["data"] = np.frombuffer(buf, dtype=np.int32).reshape(self.out_shape).copy()
        return out

    def close(self) -> None:
        if self.handle:
            _check(load().xcorr_stream_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BDI:
    """Baseline-dependent integration over a plan: one cadence per 128 x 128
    tile pair; ``step()`` after each base integration returns the due tile
    pairs as dense int32 [n_due][C][128][128][2] blocks (on the device)."""

    def __init__(self, plan: "Plan", cadence):
        torch = plan._torch
        self.plan, self._torch = plan, torch
        cad = [int(c) for c in cadence]
        self.n_tp = len(cad)
        arr = (ctypes.c_int * self.n_tp)(*cad)
        self.handle = ctypes.c_void_p()
        _check(load().xcorr_bdi_create(ctypes.byref(self.handle), plan.handle, arr, self.n_tp))

    def step(self, stream=None):
        """(blocks tensor [n_due][C][128][128][2], due tile pairs, their sample counts)."""
        torch = self._torch
        n = ctypes.c_int()
        due = (ctypes.c_int * self.n_tp)()
        smp = (ctypes.c_int64 * self.n_tp)()
        out = torch.empty((self.n_tp, self.plan.n_channels, 128, 128, 2), dtype=torch.int32, device="cuda")
        _check(load().xcorr_bdi_step(self.handle, out.data_ptr(), 1, self.plan._stream(stream),
                                     ctypes.byref(n), due, smp))
        k = n.value
        return out[:k], list(due[:k]), list(smp[:k])

    def close(self) -> None:
        if self.handle:
            load().xcorr_bdi_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Several 4+4-bit correlations of uneven size in one tensor-core launch.

    ``subarrays`` lists (n_stations, n_channels, n_time); ``execute(inputs)``
    takes one CUDA tensor per subarray and returns the int32 [C][P][2] outputs.
    """

    def __init__(self, subarrays: list[tuple[int, int, int]]):
        import torch
        self._torch = torch
        self.subarrays = list(subarrays)
        self.handle = xcorr_batch_create(self.subarrays)
        self.outputs = [torch.empty((nc, (2 * ns) * (2 * ns + 1) // 2, 2), dtype=torch.int32,
                                    device="cuda") for ns, nc, _ in self.subarrays]

    def _stream(self, stream) -> int:
        if stream is None:
            return self._torch.cuda.current_stream().cuda_stream
        return getattr(stream, "cuda_stream", stream)

    def set_variant(self, stage_variant: int) -> None:
        xcorr_batch_set_variant(self.handle, stage_variant)

    def set_subarray_variants(self, variants: list[int]) -> None:
        xcorr_batch_set_subarray_variants(self.handle, list(variants))

    def subarray_variants(self) -> list[int]:
        return xcorr_batch_get_subarray_variants(self.handle, len(self.subarrays))

    def autotune(self, inputs, stream=None) -> list[int]:
        """Per subarray, the fused shape that runs it fastest (or the cached one);
        overwrites the outputs."""
        return xcorr_batch_autotune(self.handle, [x.data_ptr() for x in inputs],
                                    [o.data_ptr() for o in self.outputs], self._stream(stream))

    def execute(self, inputs, stream=None):
        xcorr_batch_execute(self.handle, [x.data_ptr() for x in inputs],
                            [o.data_ptr() for o in self.outputs], self._stream(stream))
        return self.outputs

    def capture(self, inputs, stream=None) -> None:
        self._captured = list(inputs)  # the graph reads these buffers
        xcorr_batch_capture(self.handle, [x.data_ptr() for x in inputs],
                            [o.data_ptr() for o in self.outputs], self._stream(stream))

    def replay(self, stream=None):
        xcorr_batch_replay(self.handle, self._stream(stream))
        return self.outputs

    def sync(self, stream=None) -> None:
        xcorr_batch_sync(self.handle, self._stream(stream))

    def close(self) -> None:
        if self.handle is not None:
            xcorr_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """A plan with PyTorch tensors for device memory and streams.

    ``execute(x)`` takes a CUDA tensor in the plan's input layout
    (uint8 [t][c][s][2] for CI4, int8 [t][c][s][2][2] for CI8, float32
    [t][c][s][2][2] for CF32); ``dump()`` returns the packed-triangle
    visibilities as a [C][P][2] tensor, int32 (float32 for CF32; int64 /
    float64 with ``wide=True``), or writes them into ``out``.
    """

    def __init__(self, n_stations: int, n_channels: int, max_time_per_exec: int,
                 fmt: str = "ci4", engine: str = "auto", hbm_budget_bytes: int = 0):
        import torch  # device memory and streams only
        self._torch = torch
        self.fmt = fmt
        self.handle = xcorr_plan_create(n_stations, n_channels, max_time_per_exec,
                                        FORMATS[fmt], ENGINES[engine], hbm_budget_bytes)
        self.info = xcorr_plan_query(self.handle)
        self.n_stations = n_stations
        self.n_channels = n_channels

    def _out_dtype(self, wide: bool):
        torch = self._torch
        if self.fmt == "cf32":
            return torch.float64 if wide else torch.float32
        return torch.int64 if wide else torch.int32

    def set_tuning(self, stage_variant: int = 0, groups: int = 0, x_streams: int = 2,
                   unfused: int = 0) -> None:
        xcorr_plan_set_tuning(self.handle, stage_variant, groups, x_streams, unfused)

    def autotune(self, x, stream=None, cached: bool = False):
        """Time every launch shape on x and keep the fastest: (shape, ms); with
        cached=True through the process's tuning cache: (shape, ms, from_cache)."""
        if cached:
            return xcorr_autotune_cached(self.handle, x.data_ptr(), x.shape[0], self._stream(stream))
        return xcorr_autotune(self.handle, x.data_ptr(), x.shape[0], self._stream(stream))

    def _stream(self, stream) -> int:
        if stream is None:
            return self._torch.cuda.current_stream().cuda_stream
        return getattr(stream, "cuda_stream", stream)

    def execute(self, x, n_time: int | None = None, stream=None) -> None:
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous CUDA tensor")
        xcorr_execute(self.handle, x.data_ptr(), x.shape[0] if n_time is None else n_time,
                      self._stream(stream))

    def dump(self, out=None, reset: bool = True, wide: bool = False, stream=None):
        torch = self._torch
        shape = (self.n_channels, self.info["n_pairs"], 2)
        if out is None:
            out = torch.zeros(shape, dtype=self._out_dtype(wide), device="cuda")
        flags = (XCORR_DUMP_RESET if reset else 0) | (XCORR_DUMP_ADD_WIDE if wide else 0)
        self.samples = xcorr_dump(self.handle, out.data_ptr(), out.is_cuda, flags,
                                  self._stream(stream))
        return out

    def accum_load(self, src, n_samples: int, stream=None):
        """Resume an integration from a dump taken with reset=False: src is that dump (a host or
        CUDA tensor in the plan's output layout) and n_samples the samples it integrates."""
        if (not src.is_contiguous() or src.numel() != self.n_channels * self.info["n_pairs"] * 2
                or src.dtype != self._out_dtype(False)):
            raise ValueError("src must be a contiguous [C][P][2] dump of this plan, in its dtype")
        xcorr_accum_load(self.handle, src.data_ptr(), src.is_cuda, n_samples, self._stream(stream))
        self.samples = n_samples

    def execute_dump(self, x, out=None, reset: bool = True, wide: bool = False, stream=None):
        """execute(x) then dump(...), fused into one pass when x is the whole integration."""
        torch = self._torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous CUDA tensor")
        if out is None:
            out = torch.zeros((self.n_channels, self.info["n_pairs"], 2),
                              dtype=self._out_dtype(wide), device="cuda")
        flags = (XCORR_DUMP_RESET if reset else 0) | (XCORR_DUMP_ADD_WIDE if wide else 0)
        self.samples = xcorr_execute_dump(self.handle, x.data_ptr(), x.shape[0], out.data_ptr(),
                                          out.is_cuda, flags, self._stream(stream))
        return out

    def execute_dump_host(self, x, out=None, n_groups: int = 0, stream=None):
        """One integration from host memory to host memory, copies overlapped with
        the X-stage: x is a CPU tensor in the input layout (pin it for overlap);
        returns (or fills) a CPU [C][P][2] tensor.  Complete after sync()."""
        torch = self._torch
        if x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous host tensor")
        if out is None:
            out = torch.empty((self.n_channels, self.info["n_pairs"], 2), dtype=self._out_dtype(False),
                              pin_memory=True)
        xcorr_execute_dump_host(self.handle, x.data_ptr(), x.shape[0], out.data_ptr(), n_groups,
                                self._stream(stream))
        self.samples = x.shape[0]
        return out

    def sync(self, stream=None) -> None:
        xcorr_sync(self.handle, self._stream(stream))

    def query(self) -> dict:
        return xcorr_plan_query(self.handle)

    def close(self) -> None:
        if self.handle is not None:
            xcorr_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
