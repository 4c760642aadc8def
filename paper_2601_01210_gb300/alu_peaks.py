"""Measured instruction rates of the filter kernels' arithmetic on the current GPU.

Runs the microbenchmark in ``peaks/alu_peaks.cu`` (libalupeaks.so): FP32 FMA,
two-lane FP32 FMA, ex2.approx.ftz.f32, ex2.approx.f16x2, dp4a and the mixed
loop of the paired expanded filter form (2 dp4a + 1 two-lane FMA + 2 ex2 + 2
two-lane FMA per pair of taps). Each rate is given per second and per SM per
clock (the SM clock sampled by nvidia-smi while the kernels run), and the tap
peaks of the filter forms follow from them:

  taps/s = SMs x clock x min(issue bound, FMA-pipe bound, ex2 bound)

  * issue bound: 128 thread-instructions per SM and clock (4 schedulers x 32
    lanes) divided by the form's thread-instructions per tap;
  * FMA-pipe bound: the measured FMA (or two-lane FMA) rate divided by the
    form's FMA instructions per tap;
  * ex2 bound: the measured ex2 rate divided by the form's ex2 per tap.

dp4a issues to the same pipe as the two-lane FMA: the paired form's FMA-pipe
bound adds the two instructions' times per tap (two-lane FMA per tap / its
rate + dp4a per tap / its rate). On the GB300 the mixed loop of the paired
form runs at 96 % of that bound and at 71 % of the bound the two pipes would
give if they were apart.

Usage: ``python -m paper_2601_01210_gb300.alu_peaks [--out FILE]``.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import sys
import threading
import time

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libalupeaks.so")

OPS = {"ffma": 0, "ffma2": 1, "ex2_f32": 2, "ex2_f16x2": 3, "tap_paired": 4, "red_shared_f32": 5, "hfma2": 6,
       "tap_fp16": 7, "dp4a": 8}
ISSUE_PER_SM_CLK = 128.0   # 4 schedulers x one 32-lane warp instruction per clock
# per tap of each filter form: FP32 FMA-pipe thread-instructions (fma), two-lane FMA (fma2), ex2 and
# dp4a thread-instructions
FORMS = {
    "fp32": {"fma": 9.0, "fma2": 0.0, "ex2": 1.0},                 # difference form: 3 sub, 3 fma, 1 fma, 2 fma
    "fp32_expanded": {"fma": 5.0, "fma2": 0.0, "ex2": 1.0},        # 3 fma exponent, 2 fma sums
    # per tap: one dp4a (colour dot product), half a two-lane fma (exponent), one two-lane fma (sums)
    "fp32_expanded_pairs": {"fma": 0.0, "fma2": 1.5, "ex2": 1.0, "dp4a": 1.0},
    # sparse (a warp walks the observed positions of its block's footprint; per evaluated pixel and
    # position): row offset, squared distance, 4 fma exponent, 2 sums, half the column terms of the
    # two pixels a lane owns; window test (max, compare); half of the position's loads and loop work
    "fp32_sparse": {"fma": 9.0, "fma2": 0.0, "ex2": 1.0, "other": 5.0},
    # the sparse form with FP16 weights (per evaluated pixel and position, half of a lane's pair):
    # FP32 row offset, window test, squared distance and its kp product, the sums (num, weight,
    # squared-depth term); half of the pair's half2 differences, squares and exponent (7 half2
    # instructions) and of its ex2.approx.f16x2; packing and widening, the position's loads and
    # loop work
    "fp16_sparse": {"fma": 9.0, "fma2": 0.0, "ex2": 0.0, "ex2_h2": 0.5, "hfma2": 3.5, "other": 5.5},
}


def _lib():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2601_01210_gb300.build")
    L = C.CDLL(LIB_PATH)
    L.alu_peak_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_int)]
    L.alu_peak_run.restype = C.c_int
    return L


def run_op(name, blocks_per_sm=6, iters=1500, reps=5):
    """(units per second, SM count) of one operation: thread-instructions, or taps for the mixed loop."""
    ms, units, sms = C.c_double(), C.c_double(), C.c_int()
    rc = _lib().alu_peak_run(OPS[name], blocks_per_sm, iters, reps, C.byref(ms), C.byref(units), C.byref(sms))
    if rc != 0:
        raise RuntimeError(f"alu_peak_run({name}) failed with CUDA error {rc}")
    return units.value / (ms.value * 1e-3), sms.value


class _Clocks:
    """nvidia-smi SM clock samples every 100 ms while the kernels run."""

    def __init__(self, index=0):
        self.samples, self.proc = [], None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", "--query-gpu=clocks.sm,clocks.max.sm",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            try:
                sm, mx = (float(x) for x in line.split(","))
                self.samples.append((sm, mx))
            except ValueError:
                pass

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        sm = sorted(s for s, _ in self.samples)
        return (sm[len(sm) // 2] if sm else None), (self.samples[-1][1] if self.samples else None), len(sm)


def tap_peaks(rates_per_sm_clk):
    """Tap bounds per SM and clock of each filter form from the measured per-SM-per-clock rates.
    The FP16 form mixes half2, conversion and FP32 instructions whose pipes are not all measured
    apart: its peak is the measured rate of its own tap loop."""
    out = {}
    if "tap_fp16" in rates_per_sm_clk:
        out["fp16"] = {"taps_per_sm_clk": rates_per_sm_clk["tap_fp16"], "binds": "measured_tap_loop",
                       "bounds_taps_per_sm_clk": {"measured_tap_loop": round(rates_per_sm_clk["tap_fp16"], 3)},
                       "thread_instructions_per_tap": None}
    for form, k in FORMS.items():
        instr = (k["fma"] + k["fma2"] + k["ex2"] + k.get("ex2_h2", 0.0) + k.get("hfma2", 0.0) + k.get("dp4a", 0.0) +
                 k.get("lds", 0.0) + k.get("red", 0.0) + k.get("other", 0.0))
        bounds = {"issue": ISSUE_PER_SM_CLK / instr}
        if k["ex2"]:
            bounds["ex2"] = rates_per_sm_clk["ex2_f32"] / k["ex2"]
        if k.get("ex2_h2"):
            bounds["ex2"] = rates_per_sm_clk["ex2_f16x2"] / k["ex2_h2"]
        if k.get("dp4a") and "dp4a" not in rates_per_sm_clk:
            continue
        if k.get("red"):
            if "red_shared_f32" not in rates_per_sm_clk:
                continue
            bounds["smem_atomic"] = rates_per_sm_clk["red_shared_f32"] / k["red"]
        if k["fma"]:   # with the form's half2 FMAs on the same pipe
            bounds["fma_pipe"] = 1.0 / (k["fma"] / rates_per_sm_clk["ffma"] +
                                        k.get("hfma2", 0.0) / rates_per_sm_clk.get("hfma2", 1.0))
        if k["fma2"]:   # with the form's dp4a on the same pipe
            bounds["fma_pipe"] = 1.0 / (k["fma2"] / rates_per_sm_clk["ffma2"] +
                                        k.get("dp4a", 0.0) / rates_per_sm_clk.get("dp4a", 1.0))
        binding = min(bounds, key=bounds.get)
        out[form] = {"taps_per_sm_clk": bounds[binding], "binds": binding,
                     "bounds_taps_per_sm_clk": {b: round(v, 3) for b, v in bounds.items()},
                     "thread_instructions_per_tap": instr}
    return out


def measure(device_index=0, warm_s=0.5):
    """Rates of every operation on the current device, the sampled SM clock and the tap peaks."""
    clocks = _Clocks(device_index)
    t_end = time.perf_counter() + warm_s
    while time.perf_counter() < t_end:   # bring the clock up before the timed launches
        run_op("ffma", reps=2)
    rates, sms = {}, None
    for name in OPS:
        best = 0.0
        for _ in range(3):
            r, sms = run_op(name)
            best = max(best, r)
        rates[name] = best
    sm_mhz, sm_max, n = clocks.stop()
    clk = (sm_mhz or sm_max or 2070.0) * 1e6
    per = {k: v / (sms * clk) for k, v in rates.items()}
    peaks = tap_peaks(per)
    for form, p in peaks.items():
        p["taps_per_s"] = p["taps_per_sm_clk"] * sms * clk
    return {
        "what": "instruction rates of the filter kernels' arithmetic: best of 3 x 5 launches of "
                f"{sms} x 6 blocks of 256 threads, 8 independent chains per thread (CUDA events)",
        "sms": sms, "sm_mhz_median": sm_mhz, "sm_max_mhz": sm_max, "clock_samples": n,
        "units": "thread-instructions (taps for tap_paired)",
        "rate_per_s": {k: round(v, 1) for k, v in rates.items()},
        "rate_per_sm_clk": {k: round(v, 3) for k, v in per.items()},
        "tap_peaks": peaks,
        "tap_paired_measured_taps_per_sm_clk": round(per["tap_paired"], 3),
    }


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(a.device)
    res = measure(a.device)
    res["gpu"] = torch.cuda.get_device_name(a.device)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main(sys.argv[1:])
