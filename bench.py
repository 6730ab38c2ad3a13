#!/usr/bin/env python3
"""Benchmark: rigid-body force/torque evaluation, bead sum vs pair network.

Workload: 32768 cubes (5x5x5 beads, LJ eps = sigma = 1, r_c = 2.5), packing
fraction 0.20, seeded lattice placement, random orientations, Maxwell
velocities at kT = 1, NVE velocity Verlet at dt = 0.002.

One bench step = one full MD step (integrate, cell list, pair list, pair
force/torque evaluation, per-body reduction and half kick) of the same system
on each force path: the bead double sum (FP32), the pair network at FP32
accuracy (tensor cores, split FP16 operands: RB_F16X3) and the pair network in
BF16 (tensor cores).  The headline `value` is the BF16 network path's
body-pair force+torque evaluations per second (its MD steps/s are in `paths`
with the other two, the bead sum being the comparison and the reference of
the model error reported beside it); the SIMT FP32 network kernel is timed beside
them (`nn_fp32_simt`).  The arithmetic peaks the rooflines divide by are
measured here by register-resident probes (rb_peak_probe) with the SM clock
sampled during them.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
system stream; a 256 MiB buffer is written between steps (outside the events)
so that every step starts with a cold L2.  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same body pairs instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair force+torque evals/s & MD steps/s, NN vs bead-sum on GB300 at fixed error"
UNIT = "pair evals/s"
N_BODIES, PHI, SEED, KT, DT = 32768, 0.20, 3, 1.0, 0.002
WIDTH, DEPTH = 128, 3

# DRAM bytes (read + write) per launch of each pair kernel at this workload,
# from ncu (dram__bytes_read.sum + dram__bytes_write.sum, median over the
# captured launches of the same kernel code) on
#   python bench.py --steps 3 --warmup 3 --no-cpu-baseline --no-serving --train-steps 0
#                   --drift-steps 0 --no-paper-workload --fnet-train-steps 0
#                   --descriptor-comparison 0
# None marks a kernel not captured since it last changed.
NCU_DRAM_BYTES = {"k_bead_pairs": 1.869e6, "k_nn_f32": 2.185e6, "k_nn_tc2p": 2.052e6,
                  "k_nn_tc256": 2.474e6, "k_nn_f16x3": 2.213e6}
# The MD step's HBM-side kernels from the same captures (median launch, no
# list rebuild due): DRAM bytes read + written and the ncu duration (cold L2,
# serialised: the events inside the captured step graph cannot time single
# kernels).  Algorithmic bytes: the reduction reads 48 B per neighbour entry
# and 64 B per body and writes 64 B per body; the integrator reads and writes
# 64 B per body.
NCU_STEP_KERNELS = {"k_reduce": {"dram_bytes": 10.896e6, "ncu_us": 6.2},
                    "k_integrate_first": {"dram_bytes": 3.706e6, "ncu_us": 5.3}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--paths", default="beads,nn_f16x3,nn_bf16")
    ap.add_argument("--cpu-sample-pairs", type=int, default=100000)
    ap.add_argument("--ref-sample-pairs", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-steps", type=int, default=40000)
    ap.add_argument("--train-samples", type=int, default=1000000)
    ap.add_argument("--train-lr", type=float, default=3e-3)
    ap.add_argument("--train-f-scale", type=float, default=2.0)
    ap.add_argument("--no-symmetry", action="store_true")
    ap.add_argument("--train-contact", type=float, default=0.85)
    ap.add_argument("--train-cutoff-width", type=float, default=1.0)
    ap.add_argument("--train-lam-e", type=float, default=0.1)
    ap.add_argument("--cyl-train-steps", type=int, default=12000)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--descriptor-comparison", type=int, default=1)
    ap.add_argument("--no-paper-workload", action="store_true")
    ap.add_argument("--fnet-train-steps", type=int, default=20000)
    ap.add_argument("--paper-nn-train-steps", type=int, default=30000)
    ap.add_argument("--serving-requests", type=int, default=256)
    ap.add_argument("--serving-steps", type=int, default=1000)
    ap.add_argument("--serving-nmax", type=int, default=65536)
    ap.add_argument("--skin", type=float, default=0.4)
    ap.add_argument("--large-system", type=int, default=524288,
                    help="bodies of the larger system the BF16 kernel is also timed on (0: skip)")
    ap.add_argument("--drift-steps", type=int, default=10000)
    ap.add_argument("--drift-every", type=int, default=500)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(ms_step: float, units: float, device=None):
    """Max of the per-step time and sum of the work units over all ranks (no-op
    for one process).  Returns (ms_step_max, units_total)."""
    import torch

    try:
        import torch.distributed as dist

        active = dist.is_available() and dist.is_initialized()
    except Exception:
        active = False
    if not active:
        return ms_step, units
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def serving_run(api, inputs, mlp, n_requests=256, steps=1000, n_max=65536, seed=5,
                rate_factor=8.0, budget_bytes=2 << 30, slots=8, solo_rates=None, lanes=None,
                cyl_mlp=None, rho=(0.0, 0.0), alone_steps=100):
    """Serving workload: cube/cylinder replicas with N log-uniform in
    [512, n_max], phi in [0.05, 0.25], kT in [0.5, 1.5], `steps` MD steps each,
    Poisson arrivals at rate_factor / (solo run time of the first request), so
    about rate_factor replicas are in flight; cubes on the cube network (BF16),
    cylinders on the cylinder network (cyl_mlp, BF16) or, without one, on the
    bead path.  solo_rates (optional): pair evaluations/s of each path on one
    large system alone, {"nn": ..., "nn_cyl": ..., "beads": ...}; the mix's
    reference rate then weights them by each path's share of the pairs
    evaluated.  rho: the bead-fallback radii of the cube and the cylinder
    network (0: none).  alone_steps (0: skip): each request is also run alone
    on a fresh server for that many steps, one resident at a time, and its
    median step time in the mix is compared with its median step time alone."""
    import time as _t

    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_requests):
        shape = "cube" if rng.random() < 0.5 else "cylinder"
        n = int(round(math.exp(rng.uniform(math.log(512), math.log(n_max)))))
        phi = float(rng.uniform(0.05, 0.25))
        kT = float(rng.uniform(0.5, 1.5))
        M = 125.0 if shape == "cube" else 152.0
        I = [500.0] * 3 if shape == "cube" else [1234.2857142857142, 1234.2857142857142, 384.0]
        while True:
            try:
                st, L = inputs.system_state(n, phi, kT, seed * 1000 + k, M, I, shape)
                break
            except ValueError:
                phi -= 0.02
        net = mlp if shape == "cube" else cyl_mlp
        path = api.RB_PATH_NN if net is not None else api.RB_PATH_BEADS
        reqs.append((st, L, shape, path))
    # calibration: one solo request to set the arrival rate
    srv = make_server(api, budget_bytes, slots, mlp, cyl_mlp, lanes, rho)
    st, L, shape, path = reqs[0]
    t0 = _t.perf_counter()
    srv.wait(srv.submit(st, [L] * 3, shape, path, "bf16", steps, skin=0.4))
    t_solo = _t.perf_counter() - t0
    srv.close()
    gaps = rng.exponential(t_solo / rate_factor, size=n_requests)
    srv = make_server(api, budget_bytes, slots, mlp, cyl_mlp, lanes, rho)
    t0 = _t.perf_counter()
    tickets = []
    for (st, L, shape, path), g in zip(reqs, gaps):
        tickets.append(srv.submit(st, [L] * 3, shape, path, "bf16", steps, skin=0.4))
        _t.sleep(g)
    res = [srv.wait(t) for t in tickets]
    makespan = _t.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    # capacity: the same requests all submitted at once (a closed queue), so
    # the aggregate rate is the server's, not the arrival process's
    srv = make_server(api, budget_bytes, slots, mlp, cyl_mlp, lanes, rho)
    t0 = _t.perf_counter()
    tk = [srv.submit(st, [L] * 3, shape, path, "bf16", steps, skin=0.4) for st, L, shape, path in reqs]
    for t in tk:
        srv.wait(t)
    sat_span = _t.perf_counter() - t0
    sat = srv.stats()
    srv.close()
    ok = sum(r["status"] == 0 for r in res)
    alone = None
    if alone_steps > 0:
        srv = make_server(api, budget_bytes, slots, mlp, cyl_mlp, lanes, rho)
        solo_ms = []
        for st, L, shape, path in reqs:
            r = srv.wait(srv.submit(st, [L] * 3, shape, path, "bf16", alone_steps, skin=0.4))
            solo_ms.append(r["step_ms_p50"] if r["status"] == 0 and r["steps_done"] > 0 else None)
        srv.close()
        both = [(m["step_ms_p50"], a) for m, a in zip(res, solo_ms)
                if a and m["status"] == 0 and m["steps_done"] > 0]
        ratio = np.array([m / a for m, a in both])
        a_ms = np.array([a for _, a in both])
        alone = {"requests": len(both), "steps_each": alone_steps,
                 "slowdown_p50": float(np.percentile(ratio, 50)),
                 "slowdown_p99": float(np.percentile(ratio, 99)),
                 "alone_step_ms_p50": float(np.percentile(a_ms, 50)),
                 "alone_step_ms_p99": float(np.percentile(a_ms, 99)),
                 "note": "each request alone on the server (one resident at a time): slowdown = "
                         "its median step time in the mix / its median step time alone; "
                         "alone_step_ms: the spread of the requests' own step times (every "
                         "request runs the same number of steps), the p99/p50 the size mix "
                         "has with no sharing at all"}

    def path_key(shape, path, r):
        if path == api.RB_PATH_NN and not r["fell_back"]:
            return "nn" if shape == "cube" else "nn_cyl"
        return "beads"

    by_path = {"nn": 0.0, "nn_cyl": 0.0, "beads": 0.0}
    for (_, _, shape, path), r in zip(reqs, res):
        by_path[path_key(shape, path, r)] += float(r["pairs"]) * float(r["steps_done"])
    mix = None
    if solo_rates and all(solo_rates.get(k) for k in by_path if by_path[k] > 0):
        tot = sum(by_path.values())
        ref = tot / sum(v / solo_rates[k] for k, v in by_path.items() if v > 0)
        # per request: its median step time over the time its pairs take alone on the GPU
        slow = []
        for (_, _, shape, path), r in zip(reqs, res):
            key = path_key(shape, path, r)
            if r["pairs"] > 0 and solo_rates.get(key):
                slow.append(r["step_ms_p50"] / (1e3 * r["pairs"] / solo_rates[key]))
        mix = {"pairs_by_path": by_path, "solo_rates": solo_rates, "reference_rate": ref,
               "pair_rate_slowdown_p50": float(np.percentile(slow, 50)) if slow else None,
               "pair_rate_slowdown_p99": float(np.percentile(slow, 99)) if slow else None,
               "pair_rate_slowdown_note": "per request: median step time / (its pairs at its "
                                          "path's rate on one large system); a small replica's "
                                          "step has a fixed floor (its launches and list "
                                          "kernels) that this ignores, so it is large for small "
                                          "replicas: latency_vs_alone compares with each "
                                          "request's own step time alone",
               "efficiency_poisson": stats["pair_evals"] / makespan / ref,
               "efficiency_saturated": sat["pair_evals"] / sat_span / ref,
               "note": "reference_rate: the same pairs at each path's rate on one large system "
                       "alone (cubes: BF16 network, 32768-cube bench system; cylinders: the "
                       "width-256 cylinder network or the bead sum, 32768-cylinder system)"}
    return {"requests": n_requests, "completed_ok": ok, "steps_each": steps,
            "workload": f"cube or cylinder with probability 1/2, N log-uniform in [512, {n_max}], "
                        f"phi in [0.05, 0.25], kT in [0.5, 1.5]; Poisson arrivals, about "
                        f"{rate_factor:g} replicas in flight; HBM budget {budget_bytes >> 20} MiB, "
                        f"{slots} slots; cubes on the BF16 cube network, cylinders on "
                        + ("the BF16 width-256 cylinder network" if cyl_mlp is not None
                           else "the bead path")
                        + (f"; network pairs closer than {rho[0]:.3f} (cubes) / {rho[1]:.3f} "
                           f"(cylinders) sigma take the bead sum" if max(rho) > 0 else ""),
            "makespan_s": makespan, "pair_evals_per_s": stats["pair_evals"] / makespan,
            "step_ms_p50": stats["step_ms_p50"], "step_ms_p99": stats["step_ms_p99"],
            "mix_reference": mix, "latency_vs_alone": alone,
            "saturated": {"note": "all requests submitted at once: the server's capacity",
                          "makespan_s": sat_span, "pair_evals_per_s": sat["pair_evals"] / sat_span,
                          "step_ms_p50": sat["step_ms_p50"], "step_ms_p99": sat["step_ms_p99"]},
            "peak_resident": stats["peak_resident"], "solo_calibration_s": t_solo,
            "fell_back": sum(r["fell_back"] for r in res),
            "max_rel_energy_drift": max(abs(r["e_end"] - r["e_start"]) / (r["n_bodies"])
                                        for r in res)}


def make_server(api, budget_bytes, slots, mlp, cyl_mlp, lanes, rho=(0.0, 0.0)):
    """A server whose network-path cubes use `mlp` and cylinders `cyl_mlp`,
    with the bead-fallback radii rho = (cube, cylinder)."""
    srv = api.Server(budget_bytes, slots, mlp, steps_per_tick=8, lanes=lanes)
    if mlp is not None:
        srv.set_network("cube", mlp, rho_min=rho[0])
    if cyl_mlp is not None:
        srv.set_network("cylinder", cyl_mlp, rho_min=rho[1])
    return srv


def path_info_rate(per_path_ms, n_pairs, p):
    """Pair evaluations/s of one timed path of the MD step (None if not run)."""
    if p not in per_path_ms:
        return None
    return n_pairs[p] / (statistics.mean(per_path_ms[p]) * 1e-3)


def make_inputs(rank=0):
    from paper_2402_12199_gb300 import inputs

    # cube: 125 beads of unit mass, principal moments 500 (5x5x5 lattice at 1 sigma)
    st, L = inputs.system_state(N_BODIES, PHI, KT, SEED + 1000 * rank, 125.0, [500.0] * 3, "cube")
    mu, isd = inputs.feature_normalisation(5.0, 4 * math.sqrt(3) + 2.5)
    flat = inputs.mlp_params(WIDTH, DEPTH, 5, mu=mu, inv_sd=isd)
    return st, L, flat


def gpu_uuid(local: int):
    """NVML name of the CUDA device (GPU-<uuid>), or None."""
    try:
        import torch

        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # NVML clock-event reason bits (nvml.h): the four reported by name
    NVML_REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
                    0x4: "sw_power_cap"}

    def __init__(self, index: int, uuid: str = None):
        self.index = index
        self.uuid = uuid
        self.p = None
        self.nv = []  # (sm MHz, max sm MHz, reason bits) read through NVML
        self._stop = None

    def _nvml_handle(self):
        """Read-only NVML handle of this GPU (by UUID, else by index), or None."""
        import ctypes

        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None, None
            h = ctypes.c_void_p()
            ok = False
            if self.uuid:
                ok = lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h)) == 0
            if not ok:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h)) == 0
            return (lib, h) if ok else (None, None)
        except (OSError, AttributeError):
            return None, None

    def _poll(self):
        """Clock samples every half millisecond while the timed region runs
        (nvidia-smi's own loop cannot sample a region of a few milliseconds)."""
        import ctypes

        lib, h = self._nvml_handle()
        if lib is None:
            return
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
        mhz, mx, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and  # NVML_CLOCK_SM
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0):
                bits = r.value if reasons_fn and reasons_fn(h, ctypes.byref(r)) == 0 else 0
                self.nv.append((float(mhz.value), float(mx.value), int(bits)))
            time.sleep(0.0005)

    def __enter__(self):
        import threading

        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._poll, daemon=True)
        self._t.start()
        t0 = time.perf_counter()  # the poller is reading before the region starts
        while not self.nv and self._t.is_alive() and time.perf_counter() - t0 < 2.0:
            time.sleep(0.0005)
        return self

    def __exit__(self, *a):
        self.out = ""
        self._stop.set()
        self._t.join(timeout=5)
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], [], set()
        for mhz, mx, bits in self.nv:
            sm.append(mhz)
            smax.append(mx)
            for b, n in self.NVML_REASONS.items():
                if bits & b:
                    reasons.add(n)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "sources": {"nvml_polls": len(self.nv), "nvidia_smi": len(sm) - len(self.nv)}}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def measure_unit_peaks(api, torch, local: int) -> dict:
    """Throughput of FFMA, FFMA2 and the MUFU ex2 / rcp / tanh, measured by
    rb_peak_probe: each kind calibrated to about 0.2 s per launch, then five
    launches timed with CUDA events while nvidia-smi samples the SM clock.
    Rates in operations/s (FMA probes: FMAs/s, reported as TFLOP/s = 2 FMA)
    and per SM per clock at the median sampled clock."""
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    out = {}
    with Clocks(local, gpu_uuid(local)) as clk:
        for kind in ("ffma", "ffma2", "ex2", "rcp", "tanh"):
            iters = 2000
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            api.peak_probe(kind, 4, iters)
            b.record(stream)
            torch.cuda.synchronize()
            iters = max(iters, int(iters * 200.0 / max(a.elapsed_time(b), 1e-3)))
            ops = 0.0
            a.record(stream)
            for _ in range(5):
                ops += api.peak_probe(kind, 4, iters)
            b.record(stream)
            torch.cuda.synchronize()
            out[kind] = ops / (a.elapsed_time(b) * 1e-3)
    c = clk.summary()
    mhz = c["sm_mhz"] or 2070.0
    res = {"ffma_tflops": 2 * out["ffma"] / 1e12, "ffma2_tflops": 2 * out["ffma2"] / 1e12,
           "ex2_gops": out["ex2"] / 1e9, "rcp_gops": out["rcp"] / 1e9, "tanh_gops": out["tanh"] / 1e9,
           "per_sm_per_clock": {k: v / (sms * mhz * 1e6) for k, v in out.items()},
           "clock": c, "sms": sms,
           "how": "rb_peak_probe: 4 CTAs of 256 threads per SM, 8 independent register chains "
                  "per thread, 5 launches of ~0.2 s timed with CUDA events; per_sm_per_clock "
                  "uses the median SM clock sampled during the probes"}
    res["fp32_tflops"] = max(res["ffma_tflops"], res["ffma2_tflops"])
    return res


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def bead_flops_per_pair(n_beads: int) -> float:
    # every bead-pair distance: 3 subtractions + 1 multiply + 2 FMA = 8 flops
    return 8.0 * n_beads * n_beads


def _qmat_rows(q):
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)],
                    -2)


def bead_work(s, box, rc: float, n_sample: int = 2000, seed: int = 0) -> dict:
    """The work the bead-sum kernel has to do on a system's current pair list.
    Columns of body i's template (beads sharing x, y) whose segment lies
    farther than r_c + r_circ from body j's centre are never tested, so the
    distance tests are (columns left) x (beads per column) x n_j per pair, 8
    flop each; plus 16 flop per bead pair within r_c (counted on a sample of
    pairs) and 18 flop per bead of j rotated into i's frame (pairs with a
    column left)."""
    tmpl = s.template().astype(np.float64)
    n = len(tmpl)
    st = s.get_state(to_host=True)
    pos = st["pos"][:, :3].astype(np.float64)
    R = _qmat_rows(st["quat"].astype(np.float64))
    pairs = s.pairs().astype(np.int64)
    box = np.asarray(box, dtype=np.float64)
    d = pos[pairs[:, 1]] - pos[pairs[:, 0]]
    d -= box * np.rint(d / box)
    sb = np.einsum("pki,pk->pi", R[pairs[:, 0]], d)  # R_i^T d
    xy, inv = np.unique(np.round(tmpl[:, :2], 6), axis=0, return_inverse=True)
    inv = inv.ravel()
    cnt = np.bincount(inv, minlength=len(xy))
    zlo = np.array([tmpl[inv == c, 2].min() for c in range(len(xy))])
    zhi = np.array([tmpl[inv == c, 2].max() for c in range(len(xy))])
    r_circ = float(np.sqrt((tmpl ** 2).sum(1)).max())
    dz = np.maximum(np.maximum(zlo[None] - sb[:, 2:3], sb[:, 2:3] - zhi[None]), 0.0)
    dist2 = (sb[:, 0:1] - xy[None, :, 0]) ** 2 + (sb[:, 1:2] - xy[None, :, 1]) ** 2 + dz ** 2
    kept = dist2 <= (rc + r_circ) ** 2
    tests = float((kept * cnt[None]).sum()) * n
    rotated = float(kept.any(1).sum()) * n
    rng = np.random.default_rng(seed)
    sel = rng.choice(len(pairs), size=min(n_sample, len(pairs)), replace=False)
    n_in = 0
    for a in range(0, len(sel), 64):
        p = pairs[sel[a:a + 64]]
        bi = np.einsum("pij,kj->pki", R[p[:, 0]], tmpl)
        bj = np.einsum("pij,kj->pki", R[p[:, 1]], tmpl) + d[sel[a:a + 64]][:, None, :]
        r2 = ((bj[:, None, :, :] - bi[:, :, None, :]) ** 2).sum(-1)
        n_in += int((r2 < rc * rc).sum())
    n_in_total = n_in / len(sel) * len(pairs)
    flops = 8.0 * tests + 16.0 * n_in_total + 18.0 * rotated
    return {"flops": flops, "pairs": len(pairs), "distance_tests_per_pair": tests / len(pairs),
            "columns_left_per_pair": float(kept.sum(1).mean()), "columns": len(xy),
            "n_in_per_pair": n_in_total / len(pairs),
            "brute_force_flops": bead_flops_per_pair(n) * len(pairs)}


def nn_flops_per_pair(width: int, depth: int) -> float:
    # forward GEMMs (10 -> w, (depth-1) x w -> w, w -> 1) and the same again backward
    fwd = 2 * (10 * width + (depth - 1) * width * width + width)
    return 2.0 * fwd


_PAIR_CACHE = {}


def cpu_baseline(st, L, flat, n_sample):
    """FP64 oracle (single thread) on a bounded sample of the workload's pairs."""
    import oracle
    from oracle import bodies, nn

    tmpl = bodies.cube_template()
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    Rc = bodies.pair_cutoff(tmpl)
    key = (id(st), n_sample)
    if key not in _PAIR_CACHE:
        allp = oracle.pairs_bruteforce(pos, box, Rc)
        rng = np.random.default_rng(0)
        _PAIR_CACHE[key] = allp[np.sort(rng.choice(len(allp), min(n_sample, len(allp)),
                                                   replace=False))]
    pairs = _PAIR_CACHE[key]
    t0 = time.perf_counter()
    oracle.forces_beads(pos, quat, box, tmpl, pairs)
    t_bead = time.perf_counter() - t0
    import torch

    torch.set_num_threads(1)
    p = nn.unpack(np.asarray(flat, np.float64), WIDTH, DEPTH)
    t0 = time.perf_counter()
    nn.forces_nn(p, pos, quat, box, pairs)
    t_nn = time.perf_counter() - t0
    return {"bead_pairs_per_s": len(pairs) / t_bead, "nn_pairs_per_s": len(pairs) / t_nn,
            "pairs": int(len(pairs)), "t_bead_s": t_bead, "t_nn_s": t_nn}


_CPU_STATE = {}


def _cpu_worker_init(pos, quat, box, flat):
    import torch

    from oracle import bodies, nn

    torch.set_num_threads(1)
    _CPU_STATE.update(pos=pos, quat=quat, box=box, tmpl=bodies.cube_template(),
                      p=nn.unpack(np.asarray(flat, np.float64), WIDTH, DEPTH))


def _cpu_worker_ping(_):
    return os.getpid()


def _cpu_worker_pairs(pairs):
    import oracle
    from oracle import nn

    c = _CPU_STATE
    oracle.forces_beads(c["pos"], c["quat"], c["box"], c["tmpl"], pairs)
    nn.forces_nn(c["p"], c["pos"], c["quat"], c["box"], pairs)
    return len(pairs)


def cpu_baseline_parallel(st, L, flat, n_sample, workers):
    """The same oracle calls on the same sample, split into chunks over a pool
    of `workers` processes (started with spawn, after the GPU work): a timing
    wrapper only, the oracle code is unchanged."""
    import multiprocessing as mp

    cpu_baseline(st, L, flat, n_sample)  # fills the sample cache
    pairs = _PAIR_CACHE[(id(st), n_sample)]
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    chunks = np.array_split(pairs, 4 * workers)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_cpu_worker_init,
                  initargs=(pos, quat, np.array([L] * 3), flat)) as pool:
        pool.map(_cpu_worker_ping, range(4 * workers))  # workers up and initialised
        t0 = time.perf_counter()
        done = sum(pool.map(_cpu_worker_pairs, chunks, chunksize=1))
        t = time.perf_counter() - t0
    return {"value": 2 * done / t, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"the same {done} body pairs, bead sum and network, in {len(chunks)} "
                      f"chunks over {workers} spawned processes (one thread each)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    st, L, flat = make_inputs(0)
    res = []
    for _ in range(args.warmup):
        cpu_baseline(st, L, flat, args.ref_sample_pairs)
    for _ in range(args.steps):
        r = cpu_baseline(st, L, flat, args.ref_sample_pairs)
        res.append(r)
    pairs = sum(2 * r["pairs"] for r in res)
    t = sum(r["t_bead_s"] + r["t_nn_s"] for r in res)
    v = pairs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{N_BODIES} cubes (125 beads), phi={PHI}, LJ rc=2.5, "
                                   f"MLP 10-{WIDTH}x{DEPTH}-1 SiLU; each step a sample of "
                                   f"{args.ref_sample_pairs} body pairs per path"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.ref_sample_pairs} body pairs x 2 paths per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2402_12199_gb300 import api
    from paper_2402_12199_gb300 import inputs as inputs_mod

    paths = [p for p in args.paths.split(",") if p]
    st, L, flat = make_inputs(rank)
    dev_state = {k: torch.from_numpy(st[k]).cuda() for k in ("pos", "quat", "vel", "angmom")}
    training = None
    if args.train_steps > 0 and any(p.startswith("nn") for p in paths):
        from paper_2402_12199_gb300 import train_net

        mlp, rep = train_net.train_network("cube", WIDTH, DEPTH, n_samples=args.train_samples,
                                           steps=args.train_steps, batch=4096, lr=args.train_lr,
                                           f_scale=args.train_f_scale,
                                           symmetric=not args.no_symmetry,
                                           contact=args.train_contact,
                                           cutoff_width=args.train_cutoff_width,
                                           lam_E=args.train_lam_e, time_limit_s=60.0)
        rho_fallback = rep["rho_contact_min"]
        training = {"samples": rep["samples"], "steps": rep["steps"], "batch": rep["batch"],
                    "symmetry": rep["symmetry"],
                    "sampler_pairs_per_s": (rep["samples"] + 10000) / rep["t_sample_s"],
                    "train_samples_per_s": rep["steps"] * rep["batch"] / rep["t_train_s"],
                    "train_s": rep["t_train_s"],
                    "heldout_e_F": rep["heldout_e_F"], "heldout_e_tau_i": rep["heldout_e_tau_i"],
                    "heldout_e_tau_j": rep["heldout_e_tau_j"],
                    "heldout": "10000 pairs drawn like the training set (separation uniform "
                               "from contact to Rc: dominated by contact forces)",
                    "contact": f"smallest bead-bead distance {args.train_contact} sigma "
                               "(separations reach into the repulsive wall)",
                    "loss": f"mean w (|dF_j|^2 + |dtau_i|^2 + |dtau_j|^2 + {args.train_lam_e} dE^2), "
                            f"w = 1 / (1 + |label|^2 / {args.train_f_scale}^2); FP32, Adam, lr "
                            f"{args.train_lr} with cosine decay",
                    "energy_cutoff": rep["cutoff"],
                    "nn_bead_fallback_rho": rho_fallback}
    else:
        mlp = api.MLP(WIDTH, DEPTH)
        mlp.set_params(flat)
        rho_fallback = 0.0
    stream = torch.cuda.current_stream()
    systems = {}
    for p in paths:
        s = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
        s.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
        if p.startswith("nn"):
            s.set_nn_fallback(rho_fallback)
        systems[p] = s

    def pcfg(p):
        if p == "beads":
            return dict(path=api.RB_PATH_BEADS)
        return dict(path=api.RB_PATH_NN, mlp=mlp, precision=p.split("_")[1])

    # initial forces and pair counts
    n_pairs = {}
    for p, s in systems.items():
        if p == "beads":
            s.forces_beads()
        else:
            s.forces_nn(mlp, pcfg(p)["precision"])
        n_pairs[p] = s.build_pairs()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(events):
        for p, s in systems.items():
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(1, DT, **pcfg(p))
            e1.record(stream)
            events[p].append((e0, e1))

    warm = {p: [] for p in paths}
    for _ in range(args.warmup):
        one_step(warm)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = {p: [] for p in paths}
    with Clocks(local, gpu_uuid(local)) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one_step(ev)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    path_errors = {}
    for p, s in systems.items():
        try:
            s.sync()
        except api.RBError as ex:  # reported with the path, not hidden
            path_errors[p] = str(ex)
    per_path_ms = {p: [a.elapsed_time(b) for a, b in ev[p]] for p in paths}
    # headline: the BF16 network path (the bead sum is its comparison)
    head = "nn_bf16" if "nn_bf16" in paths else paths[0]
    ms_step, pairs_all = combine_ranks(statistics.mean(per_path_ms[head]), n_pairs[head],
                                       device="cuda")
    value = pairs_all / (ms_step * 1e-3)

    # ---- measured arithmetic peaks (FFMA, FFMA2, MUFU) for the rooflines
    pk, how = peaks()
    props = torch.cuda.get_device_properties(local)
    unit = measure_unit_peaks(api, torch, local)
    burst = pk.get("bf16_tflops", 1900.0)

    # ---- the bead-sum pair kernel, timed alone with events
    roof_beads = None
    if "beads" in systems:
        s = systems["beads"]
        s.build_pairs()
        for _ in range(3):
            s.eval_pairs(api.RB_PATH_BEADS)
        durs = []
        for _ in range(10):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.eval_pairs(api.RB_PATH_BEADS)
            b.record(stream)
            durs.append((a, b))
        torch.cuda.synchronize()
        d_ms = statistics.mean(a.elapsed_time(b) for a, b in durs)
        bw = bead_work(s, [L] * 3, 2.5)
        flops = bw["flops"]
        achieved = flops / (d_ms * 1e-3) / 1e12
        peak = unit["fp32_tflops"]
        roof_beads = {"kernel": "k_bead_pairs", "bound": "alu", "achieved": achieved, "peak": peak,
                      "unit": "TFLOP/s", "frac": achieved / peak,
                      "traffic": NCU_DRAM_BYTES["k_bead_pairs"],
                      "traffic_unit": "bytes per launch (ncu)", "kernel_ms": d_ms,
                      "peak_source": "measured FP32 FMA rate (the larger of the FFMA and FFMA2 "
                                     "probes, measured_unit_peaks)",
                      "frac_of_derived_peak": achieved / fp32_peak_tflops(
                          props.multi_processor_count, pk.get("sm_max_mhz", 2070.0)),
                      "flops_per_launch": flops,
                      "work": "8 flop per bead-pair distance the column test leaves (columns of "
                              "body i within r_c + r_circ of body j's centre x their beads x the "
                              "125 beads of j) + 16 flop per bead pair within r_c + 18 flop per "
                              "bead of j rotated",
                      "work_counts": {k: v for k, v in bw.items() if k != "flops"},
                      "brute_force_equivalent_tflops": bw["brute_force_flops"] / (d_ms * 1e-3) / 1e12,
                      "note": "the kernel tests only the columns that can reach the other body, "
                              "so it does a fraction of the 125^2 distances of the brute-force "
                              "sum with the same result; brute_force_equivalent_tflops is that "
                              "sum's flops over the kernel time (context, not a fraction)"}

    roof_nn = None
    if "nn_bf16" in systems:
        s = systems["nn_bf16"]
        s.build_pairs()
        for _ in range(3):
            s.eval_pairs(api.RB_PATH_NN, mlp, "bf16")
        durs = []
        for _ in range(10):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.eval_pairs(api.RB_PATH_NN, mlp, "bf16")
            b.record(stream)
            durs.append((a, b))
        torch.cuda.synchronize()
        d_ms = statistics.mean(a.elapsed_time(b) for a, b in durs)
        np_ = n_pairs["nn_bf16"]
        # the method's flops (forward and input-gradient GEMMs) per launch
        flops = nn_flops_per_pair(WIDTH, DEPTH) * np_
        achieved = flops / (d_ms * 1e-3) / 1e12
        # tensor-core work actually issued per 128-pair tile: layer 1 one K step of
        # 16 (10 features), the input gradient's N padded to 16
        issued = 2.0 * 128 * (128 * 16 + 2 * 128 * 128 + 2 * 128 * 128 + 128 * 16) / 128 * np_
        mufu = DEPTH * WIDTH * np_ / (d_ms * 1e-3)  # one tanh.approx per SiLU evaluation
        roof_nn = {"kernel": "k_nn_tc2p", "bound": "tensor", "achieved": achieved, "peak": burst,
                   "unit": "TFLOP/s", "frac": achieved / burst, "kernel_ms": d_ms,
                   "traffic": NCU_DRAM_BYTES["k_nn_tc2p"], "traffic_unit": "bytes per launch (ncu)",
                   "peak_source": f"bf16_tflops burst ({how}; the kernel is timed alone)",
                   "flops_per_launch": flops,
                   "work": "2 x 2 (10 w + 2 w^2 + w) flop per pair (forward and input-gradient "
                           "GEMMs of the 10-128x3-1 network)",
                   "issued_tflops": issued / (d_ms * 1e-3) / 1e12,
                   "mufu": {"ops_per_pair": DEPTH * WIDTH, "achieved_gops": mufu / 1e9,
                            "peak_gops": unit["tanh_gops"], "frac": mufu / 1e9 / unit["tanh_gops"],
                            "note": "one tanh.approx per SiLU evaluation (silu' from the same "
                                    "tanh); peak = measured tanh.approx rate"}}
        # context: the same kernel and network on a system 16 times larger, where
        # the tiles fill the 304 pipelines evenly (at 98304 pairs 768 tiles take 3
        # rounds for 2.53 rounds of work)
        if world == 1 and args.large_system > 0:
            nb = args.large_system
            st_big, L_big = inputs_mod.system_state(nb, PHI, KT, SEED + 21, 125.0, [500.0] * 3,
                                                    "cube")
            sb = api.System(nb, [L_big] * 3, "cube", skin=args.skin)
            sb.set_state(*(torch.from_numpy(st_big[k]).cuda()
                           for k in ("pos", "quat", "vel", "angmom")))
            np_big = sb.build_pairs()
            for _ in range(3):
                sb.eval_pairs(api.RB_PATH_NN, mlp, "bf16")
            durs = []
            for _ in range(10):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sb.eval_pairs(api.RB_PATH_NN, mlp, "bf16")
                b.record(stream)
                durs.append((a, b))
            torch.cuda.synchronize()
            sb.sync()
            d_big = statistics.mean(a.elapsed_time(b) for a, b in durs)
            t_big = nn_flops_per_pair(WIDTH, DEPTH) * np_big / (d_big * 1e-3) / 1e12
            roof_nn["large_system"] = {
                "bodies": nb, "pairs": np_big, "kernel_ms": d_big, "achieved": t_big,
                "frac": t_big / burst, "note": "context, not the headline: the same network "
                "and kernel on a larger system of the same density"}
            del sb

    def kernel_ms(s, prec):
        s.build_pairs()
        for _ in range(3):
            s.eval_pairs(api.RB_PATH_NN, mlp, prec)
        durs = []
        for _ in range(10):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.eval_pairs(api.RB_PATH_NN, mlp, prec)
            b.record(stream)
            durs.append((a, b))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in durs)

    roof_x3 = None
    if "nn_f16x3" in systems:
        d_ms = kernel_ms(systems["nn_f16x3"], "f16x3")
        np_ = n_pairs["nn_f16x3"]
        flops = nn_flops_per_pair(WIDTH, DEPTH) * np_
        achieved = flops / (d_ms * 1e-3) / 1e12
        # three FP16 products per layer GEMM (hi.hi, hi.lo, lo.hi), the same
        # padded shapes as the BF16 kernel
        issued = 3 * 2.0 * 128 * (128 * 16 + 2 * 128 * 128 + 2 * 128 * 128 + 128 * 16) / 128 * np_
        # one ex2.approx and one rcp.approx per SiLU evaluation
        t_mufu = DEPTH * WIDTH * np_ * (1e-9 / unit["ex2_gops"] + 1e-9 / unit["rcp_gops"])
        roof_x3 = {"kernel": "k_nn_f16x3", "bound": "tensor", "achieved": achieved, "peak": burst,
                   "unit": "TFLOP/s", "frac": achieved / burst, "kernel_ms": d_ms,
                   "traffic": NCU_DRAM_BYTES["k_nn_f16x3"], "traffic_unit": "bytes per launch (ncu)",
                   "peak_source": f"bf16_tflops burst ({how}; timed alone; FP16 and BF16 share "
                                  "the dense tensor rate)",
                   "flops_per_launch": flops,
                   "work": "the network's own flops, 2 x 2 (10 w + 2 w^2 + w) per pair",
                   "issued_tflops": issued / (d_ms * 1e-3) / 1e12,
                   "issued_frac": issued / (d_ms * 1e-3) / 1e12 / burst,
                   "mufu": {"ops_per_pair": 2 * DEPTH * WIDTH, "frac": t_mufu / (d_ms * 1e-3),
                            "note": "ex2.approx + rcp.approx per SiLU evaluation against the "
                                    "measured rates of each"},
                   "note": "FP32-accurate: operands split into two scaled FP16 parts, three "
                           "tensor-core products per GEMM (issued_tflops counts them)"}

    # the SIMT FP32 network kernel, timed beside the step (a system of its own
    # when the step does not run it)
    roof_f32 = None
    simt = None
    if any(p.startswith("nn") for p in paths):
        if "nn_fp32" in systems:
            s = systems["nn_fp32"]
        else:
            s = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
            s.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
            s.set_nn_fallback(rho_fallback)
            s.forces_nn(mlp, "fp32")
            md = []
            for _ in range(3):
                s.step(1, DT, path=api.RB_PATH_NN, mlp=mlp, precision="fp32")
            for _ in range(20):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(1, DT, path=api.RB_PATH_NN, mlp=mlp, precision="fp32")
                b.record(stream)
                md.append((a, b))
            torch.cuda.synchronize()
            s.sync()
            simt = {"ms_per_md_step": statistics.mean(a.elapsed_time(b) for a, b in md),
                    "md_steps": 20, "note": "SIMT FP32 network path, same state, not in the step"}
        d_ms = kernel_ms(s, "fp32")
        n_f32 = s.build_pairs()
        flops = nn_flops_per_pair(WIDTH, DEPTH) * n_f32
        achieved = flops / (d_ms * 1e-3) / 1e12
        peak = unit["fp32_tflops"]
        roof_f32 = {"kernel": "k_nn_f32", "bound": "alu", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "kernel_ms": d_ms,
                    "traffic": NCU_DRAM_BYTES["k_nn_f32"], "traffic_unit": "bytes per launch (ncu)",
                    "peak_source": "measured FP32 FMA rate (measured_unit_peaks)",
                    "flops_per_launch": flops}
        if simt is not None:
            simt["kernel_ms"] = d_ms
            simt["f16x3_kernel_speedup"] = d_ms / roof_x3["kernel_ms"] if roof_x3 else None
            del s

    # ---- cylinder training throughput at width 256: 1M pairs drawn and
    # labelled on the device, then Adam steps on batches of 4096
    train_cyl = None
    cyl_net = None        # the trained cylinder network, kept for the serving leg
    cyl_nn_rate = None    # its pair evaluations/s on the 32768-cylinder system (no fallback)
    cyl_rho = 0.0         # its bead-fallback radius (the training set's smallest contact)
    if args.train_steps > 0 and any(p.startswith("nn") for p in paths):
        from paper_2402_12199_gb300 import train_net

        m_cyl, rc = train_net.train_network("cylinder", 256, DEPTH, n_samples=1_000_000,
                                            steps=args.cyl_train_steps, batch=4096,
                                            lr=args.train_lr, f_scale=args.train_f_scale,
                                            contact=args.train_contact, lam_E=args.train_lam_e,
                                            cutoff_width=args.train_cutoff_width, seed=4)
        # model error on an MD state of cylinders (the per-component leg's system)
        probe = api.System(8, [80.0] * 3, "cylinder")
        st_cy, L_cy = inputs_mod.system_state(32768, 0.15, KT, SEED + 11, probe.mass,
                                              probe.inertia, "cylinder")
        del probe
        s_cy = api.System(32768, [L_cy] * 3, "cylinder", skin=args.skin)
        s_cy.set_state(*(torch.from_numpy(st_cy[k]).cuda() for k in ("pos", "quat", "vel", "angmom")))
        s_cy.set_nn_fallback(rc["rho_contact_min"])
        err_cy = train_net.force_error(s_cy, m_cyl, "bf16")
        # MD steps on the network without the bead fallback, as the server runs it
        s_cy.set_nn_fallback(0.0)
        for _ in range(3):
            s_cy.step(1, DT, path=api.RB_PATH_NN, mlp=m_cyl, precision="bf16")
        ev_cy = []
        for _ in range(30):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s_cy.step(1, DT, path=api.RB_PATH_NN, mlp=m_cyl, precision="bf16")
            b.record(stream)
            ev_cy.append((a, b))
        torch.cuda.synchronize()
        s_cy.sync()
        ms_cy = statistics.mean(a.elapsed_time(b) for a, b in ev_cy)
        cyl_nn_rate = len(s_cy.pairs()) / (ms_cy * 1e-3)
        cyl_net = m_cyl
        cyl_rho = rc["rho_contact_min"]
        del s_cy
        train_cyl = {"workload": "cylinders (8 x 19 beads), network 10-256x3-1, 1M training pairs",
                     "symmetry": rc["symmetry"],
                     "sampler_pairs_per_s": (rc["samples"] + 10000) / rc["t_sample_s"],
                     "train_samples_per_s": rc["steps"] * rc["batch"] / rc["t_train_s"],
                     "steps": rc["steps"], "heldout_e_F_after_these_steps": rc["heldout_e_F"],
                     "heldout": "pairs drawn like the training set (separation uniform from "
                                "contact to Rc: dominated by contact forces)",
                     "model_error_md_state": dict(err_cy, vs="bead path on 32768 cylinders at "
                                                  "phi 0.15 (model error, not parity), BF16, "
                                                  "bead fallback below the contact separation"),
                     "ms_per_md_step": ms_cy, "pair_evals_per_s": cyl_nn_rate,
                     "md_note": "32768 cylinders at phi 0.15 on this network (k_nn_tc256), "
                                "no bead fallback"}

    # ---- network width 256 (BF16, streamed weights), same workload, timed alone
    width256 = None
    if "nn_bf16" in paths:
        m256 = api.MLP(256, DEPTH)
        mu, isd = inputs_mod.feature_normalisation(5.0, 4 * math.sqrt(3) + 2.5)
        m256.set_params(inputs_mod.mlp_params(256, DEPTH, 6, mu=mu, inv_sd=isd))
        s256 = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
        s256.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
        s256.forces_nn(m256, "bf16")
        ev256 = []
        for it in range(max(3, args.warmup) + 200):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s256.step(1, DT, path=api.RB_PATH_NN, mlp=m256, precision="bf16")
            b.record(stream)
            if it >= max(3, args.warmup):
                ev256.append((a, b))
        torch.cuda.synchronize()
        s256.sync()
        ms256 = statistics.mean(a.elapsed_time(b) for a, b in ev256)
        s256.build_pairs()
        ka = torch.cuda.Event(enable_timing=True)
        kb = torch.cuda.Event(enable_timing=True)
        ka.record(stream)
        for _ in range(10):
            s256.eval_pairs(api.RB_PATH_NN, m256, "bf16")
        kb.record(stream)
        torch.cuda.synchronize()
        k256 = ka.elapsed_time(kb) / 10
        tc256 = 2.0 * 128 * (256 * 16 + 4 * 256 * 256 + 256 * 16) / 128 * n_pairs["nn_bf16"]
        alg256 = nn_flops_per_pair(256, DEPTH) * n_pairs["nn_bf16"]
        width256 = {"ms_per_md_step": ms256, "md_steps_per_s": 1e3 / ms256,
                    "speedup_vs_beads": (statistics.mean(per_path_ms["beads"]) / ms256)
                    if "beads" in per_path_ms else None,
                    "kernel": "k_nn_tc256", "kernel_ms": k256,
                    "traffic": NCU_DRAM_BYTES["k_nn_tc256"], "traffic_unit": "bytes per launch (ncu)",
                    "tflops": alg256 / (k256 * 1e-3) / 1e12,
                    "frac_of_bf16_burst": alg256 / (k256 * 1e-3) / 1e12 / burst,
                    "issued_tflops": tc256 / (k256 * 1e-3) / 1e12,
                    "work": "2 x 2 (10 w + 2 w^2 + w) flop per pair, w = 256",
                    "steps_timed": 200}
        del s256, m256

    # ---- the paper's own workload shape: half-power half-cosine bead
    # potential (Eq. 1, continuous reading) between cubes at phi = 0.16 under
    # the Nose-Hoover thermostat (kT = 0.6, period 0.5) with dt = 0.005, bead
    # path; then the cost of one g(r) / MSD / MSR frame
    paper_wl = None
    if "beads" in paths and not args.no_paper_workload:
        KT_P, DT_P, PHI_P = 0.6, 0.005, 0.16
        stp, Lp = inputs_mod.system_state(N_BODIES, PHI_P, KT_P, SEED + 7, 125.0, [500.0] * 3, "cube")
        sp = api.System(N_BODIES, [Lp] * 3, "cube", skin=args.skin, potential="hphc",
                        hphc=inputs_mod.HPHC_PAPER)
        sp.set_state(*(torch.from_numpy(stp[k]).cuda() for k in ("pos", "quat", "vel", "angmom")))
        sp.set_thermostat(KT_P, 0.5)
        sp.forces_beads()
        sp.step(200, DT_P)  # warm-up: graph capture, list rebuilds settle
        n_pairs_p = sp.build_pairs()
        sp.set_reference()
        ev_p = []
        for _ in range(300):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sp.step(1, DT_P)
            b.record(stream)
            ev_p.append((a, b))
        torch.cuda.synchronize()
        ms_p = statistics.mean(a.elapsed_time(b) for a, b in ev_p)
        _, kt_p, kr_p = sp.energy()
        # the pair kernel alone (k_bead_pairs with the half-power half-cosine body)
        sp.build_pairs()
        kp = []
        for _ in range(10):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sp.eval_pairs(api.RB_PATH_BEADS)
            b.record(stream)
            kp.append((a, b))
        torch.cuda.synchronize()
        kms_p = statistics.mean(a.elapsed_time(b) for a, b in kp)
        hp = inputs_mod.HPHC_PAPER
        bw_p = bead_work(sp, [Lp] * 3, hp["b"] + math.pi / hp["c"])
        flops_p = bw_p["flops"]
        # analyses: one g(r) frame (pair list current) and one MSD / MSR read
        r_max_p = 0.95 * sp.pair_cutoff
        counts = sp.gr_counts(r_max_p, 200)
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        for _ in range(10):
            sp.gr_counts(r_max_p, 200, counts)
        gb.record(stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        msd_p, msr_p = sp.msd_msr()
        t_msd = time.perf_counter() - t0
        g_p = sp.gr_normalise(counts.cpu().numpy(), r_max_p, 11)
        paper_wl = {
            "workload": f"{N_BODIES} cubes (5x5x5 beads), half-power half-cosine beads of Eq. 1 "
                        f"(A=0.00035, b=1.46375, c=3.3833, p=2.5; continuous reading, cutoff "
                        f"b + pi/c), phi={PHI_P}, Nose-Hoover NVT kT={KT_P} (period 0.5), "
                        f"dt={DT_P}, skin {args.skin}",
            "ms_per_md_step": ms_p, "md_steps_per_s": 1e3 / ms_p,
            "pair_evals_per_s": n_pairs_p / (ms_p * 1e-3), "pairs": n_pairs_p,
            "steps_timed": 300, "temperature_2K_over_g": 2 * (kt_p + kr_p) / (6 * N_BODIES - 3),
            "kernel": "k_bead_pairs (half-power half-cosine)", "kernel_ms": kms_p,
            "kernel_tflops": flops_p / (kms_p * 1e-3) / 1e12,
            "frac_of_fp32_peak": flops_p / (kms_p * 1e-3) / 1e12 / unit["fp32_tflops"],
            "kernel_work": "as roofline_beads (distance tests the column test leaves, bead pairs "
                           "within the cutoff b + pi/c, rotations)",
            "kernel_work_counts": {k: v for k, v in bw_p.items() if k != "flops"},
            "gr_frame_ms": ga.elapsed_time(gb) / 10, "msd_msr_read_ms": t_msd * 1e3,
            "msd_after_300_steps": msd_p, "msr_after_300_steps": msr_p,
            "g_r_first_peak": {"r": float((np.argmax(g_p) + 0.5) * r_max_p / 200), "g": float(g_p.max())}}
        del sp
        # the network on the same workload: trained on half-power half-cosine
        # labels, BF16, same thermostat; model error against the bead sum
        if any(p.startswith("nn") for p in paths) and args.paper_nn_train_steps > 0:
            from paper_2402_12199_gb300 import train_net

            mlp_p, rep_p = train_net.train_network(
                "cube", WIDTH, DEPTH, n_samples=args.train_samples, steps=args.paper_nn_train_steps,
                batch=4096, lr=args.train_lr, lam_E=args.train_lam_e, f_scale=0.05, seed=9,
                contact=0.7, cutoff_width=args.train_cutoff_width, potential="hphc",
                hphc=inputs_mod.HPHC_PAPER, time_limit_s=40.0)
            sn = api.System(N_BODIES, [Lp] * 3, "cube", skin=args.skin, potential="hphc",
                            hphc=inputs_mod.HPHC_PAPER)
            sn.set_state(*(torch.from_numpy(stp[k]).cuda() for k in ("pos", "quat", "vel", "angmom")))
            sn.set_nn_fallback(rep_p["rho_contact_min"])
            err_p = train_net.force_error(sn, mlp_p, "bf16")
            sn.set_thermostat(KT_P, 0.5)
            sn.forces_nn(mlp_p, "bf16")
            sn.step(200, DT_P, path=api.RB_PATH_NN, mlp=mlp_p, precision="bf16")
            ev_n = []
            for _ in range(300):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sn.step(1, DT_P, path=api.RB_PATH_NN, mlp=mlp_p, precision="bf16")
                b.record(stream)
                ev_n.append((a, b))
            torch.cuda.synchronize()
            sn.sync()
            ms_n = statistics.mean(a.elapsed_time(b) for a, b in ev_n)
            _, kt_n, kr_n = sn.energy()
            paper_wl["nn_bf16"] = {
                "ms_per_md_step": ms_n, "md_steps_per_s": 1e3 / ms_n,
                "speedup_vs_beads": ms_p / ms_n,
                "temperature_2K_over_g": 2 * (kt_n + kr_n) / (6 * N_BODIES - 3),
                "model_error": dict(err_p, vs="bead path (half-power half-cosine), same state"),
                "training": {k: rep_p.get(k) for k in ("samples", "steps", "heldout_e_F", "t_train_s")},
                "net": f"10-{WIDTH}x{DEPTH}-1 SiLU, cube point group, trained on half-power "
                       f"half-cosine labels (contact 0.7 sigma, force scale 0.05)"}
            del sn, mlp_p

    # ---- per-component networks for cylinders (the paper's cylinder method):
    # 32768 cylinders at phi = 0.15, five networks (width 32, depth 3) trained
    # on the device on 1M bead-labelled pairs (capped, force-scale weighted
    # targets), then one MD
    # step per path timed on the same state, and the model error
    fnet_leg = None
    if "beads" in paths and args.fnet_train_steps > 0 and world == 1:
        from paper_2402_12199_gb300 import train_net

        Nc, PHI_C, CAP, WF, DF = 32768, 0.15, 5.0, 32, 3
        fn, rep_fn = train_net.train_fnet("cylinder", WF, DF, n_samples=1_000_000,
                                          steps=args.fnet_train_steps, batch=4096, lr=2e-3,
                                          cap=CAP, seed=8, f_scale=1.0)
        probe = api.System(8, [80.0] * 3, "cylinder")
        stc, Lc = inputs_mod.system_state(Nc, PHI_C, KT, SEED + 11, probe.mass, probe.inertia,
                                          "cylinder")
        del probe
        sysc = {}
        for pth in ("beads", "fnet"):
            sc = api.System(Nc, [Lc] * 3, "cylinder", skin=args.skin)
            sc.set_state(*(torch.from_numpy(stc[k]).cuda() for k in ("pos", "quat", "vel", "angmom")))
            sysc[pth] = sc
        err_fn = train_net.fnet_force_error(sysc["fnet"], fn)
        n_pairs_c = sysc["beads"].build_pairs()
        tc = {}
        for pth, sc in sysc.items():
            run = (lambda k, sc=sc: sc.step(k, DT)) if pth == "beads" else (lambda k, sc=sc: sc.step_fnet(fn, k, DT))
            run(20)
            evs = []
            for _ in range(100):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run(1)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
            sc.sync()
            tc[pth] = statistics.mean(a.elapsed_time(b) for a, b in evs)
        # the network pair kernel alone: whole-system forces minus nothing else
        # is not separable, so time rb_forces_fnet and rb_forces_beads (list
        # current, reduction included)
        fl = 2.0 * 5 * (4 * WF + (DF - 1) * WF * WF + WF) * n_pairs_c
        fnet_leg = {"workload": f"{Nc} cylinders (8 x 19 beads), phi={PHI_C}, NVE dt={DT}, skin "
                                f"{args.skin}; five per-component networks 4-{WF}x{DF}-1 SiLU",
                    "pairs": n_pairs_c,
                    "ms_per_md_step": {"beads": tc["beads"], "fnet": tc["fnet"]},
                    "speedup_vs_beads": tc["beads"] / tc["fnet"],
                    "fnet_pair_evals_per_s": n_pairs_c / (tc["fnet"] * 1e-3),
                    "fnet_flop_per_pair": fl / max(1, n_pairs_c),
                    "model_error": dict(err_fn, vs="bead path, same state (model error, not parity)"),
                    "training": rep_fn}
        del sysc, fn

    # ---- NVE energy conservation: a fresh copy of the workload per path, run
    # for --drift-steps steps with the FP64 total energy read every
    # --drift-every steps (outside every timed region)
    drift = None
    if args.drift_steps > 0:
        drift = {"steps": args.drift_steps, "dt": DT, "sample_every": args.drift_every,
                 "measure": "max_t |E_tot(t) - E_tot(0)| / (N kT) and the least-squares slope "
                            "per 1000 steps; E_tot = E_pot + KE_trans + KE_rot in FP64"}
        # the last entry: the BF16 network i<->j-symmetrised (each pair's energy
        # averaged over both reference bodies, whose canonical-choice
        # boundaries lie elsewhere)
        drift_runs = list(paths) + (["nn_bf16_pair_symmetrised"] if "nn_bf16" in paths else [])
        for p in drift_runs:
            sym = p.endswith("_pair_symmetrised")
            p = "nn_bf16" if sym else p
            mlp.set_pair_symmetrised(sym)
            s = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
            s.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
            if p.startswith("nn"):
                s.set_nn_fallback(rho_fallback)
            if p == "beads":
                s.forces_beads()
            else:
                s.forces_nn(mlp, pcfg(p)["precision"])
            t_series, e_series = [0], [sum(s.energy())]
            done = 0
            err = None
            try:
                while done < args.drift_steps:
                    k = min(args.drift_every, args.drift_steps - done)
                    s.step(k, DT, **pcfg(p))
                    done += k
                    t_series.append(done)
                    e_series.append(sum(s.energy()))
            except api.RBError as ex:  # e.g. bodies collapsing into one cell
                err = f"stopped after at most {done + args.drift_every} steps: {ex}"
            e = np.array(e_series)
            dev = np.abs(e - e[0]) / (N_BODIES * KT)
            finite = bool(np.all(np.isfinite(e)))
            drift[p + ("_pair_symmetrised" if sym else "")] = {
                        "max_abs_drift_per_body_kT": float(dev.max()) if finite else None,
                        "slope_per_body_kT_per_1k_steps":
                            float(np.polyfit(np.array(t_series) / 1000.0, e / (N_BODIES * KT), 1)[0])
                            if finite else None,
                        "E0_per_body_kT": float(e[0] / (N_BODIES * KT)) if finite else None,
                        "finite": finite, "steps_done": done, "error": err}
            del s
        mlp.set_pair_symmetrised(False)

    # ---- end to end through the public API with host buffers, on the
    # headline path: a client that keeps the whole velocity-Verlet state in
    # page-locked host memory (centres, orientations, momenta and the forces
    # at the current centres, one block) feeds it in, runs one MD step and
    # reads the new state and forces back into the same block, with one host
    # synchronisation per step (rb_step_host_state: rb_set_state, rb_set_forces,
    # rb_step and the copies back in one call; the forces handed back spare the
    # step an evaluation at the state it was given).
    keys4 = ("pos", "quat", "vel", "angmom")
    e2e_paths = [head]
    blk = {p: torch.empty((6, N_BODIES, 4), dtype=torch.float32).pin_memory() for p in e2e_paths}
    e2e_sys = {}
    for p in e2e_paths:
        se = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin, stream=torch.cuda.Stream())
        se.set_state(*(dev_state[k] for k in keys4))
        if p.startswith("nn"):
            se.set_nn_fallback(rho_fallback)
        se.step(1, DT, **pcfg(p))  # forces and the step graph, before the timed loop
        se.get_state(to_host=True, out={k: blk[p][i] for i, k in enumerate(keys4)})
        se.get_forces(to_host=True, out=(blk[p][4], blk[p][5]))
        e2e_sys[p] = se
    e2e_steps = max(3, min(args.steps, 50))

    def e2e_time(copies):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for p, se in e2e_sys.items():  # state and forces in, one step, both out
                se.step_host_state(blk[p], 1, DT, sync=False, copies=copies, **pcfg(p))
            torch.cuda.synchronize()
        return (time.perf_counter() - t0) / e2e_steps

    # the copy form (one copy each way around the step) for comparison, then
    # the direct form the call takes for a page-locked block (the step's
    # kernels read and write the block in host memory)
    e2e_t_copies = e2e_time(True)
    e2e_t = e2e_time(False)
    e2e_ok = all(bool(torch.isfinite(blk[p]).all()) for p in e2e_paths)
    for se in e2e_sys.values():
        se.sync()
    del e2e_sys
    h2d = len(e2e_paths) * 6 * N_BODIES * 16
    d2h = len(e2e_paths) * 6 * N_BODIES * 16
    e2e_value = sum(n_pairs[p] for p in e2e_paths) * world / e2e_t
    e2e_value_copies = sum(n_pairs[p] for p in e2e_paths) * world / e2e_t_copies

    model_error = None
    if any(p.startswith("nn") for p in paths):
        from paper_2402_12199_gb300 import train_net

        probe = api.System(N_BODIES, [L] * 3, "cube")
        probe.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
        probe.set_nn_fallback(rho_fallback)
        model_error = {"vs": "bead path, same state (model error, not parity)",
                       "trained": training is not None}
        for p in paths:
            if p.startswith("nn"):
                model_error[p] = train_net.force_error(probe, mlp, p.split("_")[1])
        # the pair-symmetrised evaluation (each pair's energy averaged over both
        # choices of reference body): its error against the bead sum, how far
        # it is from the plain evaluation (the network's i <-> j asymmetry), and
        # its MD step time, outside the timed step
        sym_prec = "f16x3" if "nn_f16x3" in paths else "fp32"
        plain = probe.forces_nn(mlp, sym_prec)
        plain_F = plain["force"][:, :3].clone()
        mlp.set_pair_symmetrised(True)
        try:
            err_sym = train_net.force_error(probe, mlp, sym_prec)
            symF = probe.forces_nn(mlp, sym_prec)["force"][:, :3]
            probe.sync()
            asym = float(torch.linalg.norm(symF - plain_F) / torch.linalg.norm(plain_F))
            sym_ms = {}
            for prec in sorted({sym_prec, "bf16"}):
                ss = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
                ss.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
                ss.set_nn_fallback(rho_fallback)
                ss.forces_nn(mlp, prec)
                for _ in range(3):
                    ss.step(1, DT, path=api.RB_PATH_NN, mlp=mlp, precision=prec)
                evs = []
                for _ in range(20):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ss.step(1, DT, path=api.RB_PATH_NN, mlp=mlp, precision=prec)
                    b.record(stream)
                    evs.append((a, b))
                torch.cuda.synchronize()
                ss.sync()
                sym_ms[prec] = statistics.mean(x.elapsed_time(y) for x, y in evs)
                del ss
            model_error["pair_symmetrised"] = {
                "precision": sym_prec, **err_sym, "asymmetry_e_F_vs_plain": asym,
                "ms_per_md_step": sym_ms,
                "note": "energy of every pair averaged over both choices of reference body "
                        "(two network passes); not in the timed step"}
        finally:
            mlp.set_pair_symmetrised(False)
        del probe
    # ---- the paper's six-number cube descriptor (SI Sec. 1) against the 10
    # features: the same training recipe and budget, then model error against
    # the bead sum on the MD state and the cost of an MD step and of the
    # network kernel, both networks timed the same way here
    desc_cmp = None
    if training is not None and args.descriptor_comparison:
        from paper_2402_12199_gb300 import train_net

        mlp6, rep6 = train_net.train_network(
            "cube", WIDTH, DEPTH, n_samples=args.train_samples, steps=args.train_steps, batch=4096,
            lr=args.train_lr, f_scale=args.train_f_scale, symmetric=True,
            contact=args.train_contact, cutoff_width=args.train_cutoff_width,
            lam_E=args.train_lam_e, time_limit_s=60.0, descriptor="paper6")

        def md_and_kernel_ms(net, prec, fb):
            sd = api.System(N_BODIES, [L] * 3, "cube", skin=args.skin)
            sd.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
            sd.set_nn_fallback(fb)
            sd.forces_nn(net, prec)
            for _ in range(3):
                sd.step(1, DT, path=api.RB_PATH_NN, mlp=net, precision=prec)
            evs = []
            for _ in range(50):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sd.step(1, DT, path=api.RB_PATH_NN, mlp=net, precision=prec)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
            sd.sync()
            md = statistics.mean(x.elapsed_time(y) for x, y in evs)
            sd.build_pairs()
            kd = []
            for _ in range(10):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sd.eval_pairs(api.RB_PATH_NN, net, prec)
                b.record(stream)
                kd.append((a, b))
            torch.cuda.synchronize()
            sd.sync()
            return md, statistics.mean(x.elapsed_time(y) for x, y in kd)

        probe6 = api.System(N_BODIES, [L] * 3, "cube")
        probe6.set_state(*(dev_state[k] for k in ("pos", "quat", "vel", "angmom")))
        desc_cmp = {"workload": "the bench state; both networks 10-128x3-1 SiLU trained with the "
                                "same recipe and time budget; model error against the bead sum",
                    "paper6": {"inputs": "p_x, p_y, p_z, alpha_1, alpha_2, alpha_3 (SI Sec. 1)",
                               "training": {k: rep6.get(k) for k in ("samples", "steps", "t_train_s",
                                                                      "heldout_e_F", "heldout_e_tau_i")}},
                    "features10": {"inputs": "s, q_rel, rho, 1/rho, rho^2 of the canonical "
                                             "configuration",
                                   "training": {k: training.get(k) for k in ("samples", "steps",
                                                                             "heldout_e_F",
                                                                             "heldout_e_tau_i")}}}
        for name, net, fb in (("paper6", mlp6, rep6["rho_contact_min"]), ("features10", mlp, rho_fallback)):
            probe6.set_nn_fallback(fb)
            for prec in ("bf16", "f16x3"):
                e = train_net.force_error(probe6, net, prec)
                md, kern = md_and_kernel_ms(net, prec, fb)
                desc_cmp[name][prec] = dict(e, ms_per_md_step=md, kernel_ms=kern)
        del probe6, mlp6

    serving = None
    if not args.no_serving and world == 1:
        solo = {"nn": path_info_rate(per_path_ms, n_pairs, "nn_bf16"), "nn_cyl": cyl_nn_rate}
        if fnet_leg is not None:
            solo["beads"] = fnet_leg["pairs"] / (fnet_leg["ms_per_md_step"]["beads"] * 1e-3)
        serving = serving_run(api, __import__("paper_2402_12199_gb300.inputs", fromlist=["x"]),
                              mlp, n_requests=args.serving_requests, steps=args.serving_steps,
                              n_max=args.serving_nmax, solo_rates=solo, cyl_mlp=cyl_net,
                              rho=(rho_fallback, cyl_rho))
        # many small replicas (where stepping them together pays most): N in
        # [512, 4096], 32 slots, about 32 in flight, the server's default lanes
        small = serving_run(api, __import__("paper_2402_12199_gb300.inputs", fromlist=["x"]),
                            mlp, n_requests=args.serving_requests, steps=args.serving_steps,
                            n_max=4096, rate_factor=32.0, budget_bytes=4 << 30, slots=32,
                            cyl_mlp=cyl_net, rho=(rho_fallback, cyl_rho))
        serving["small_replicas"] = {k: small[k] for k in
                                     ("workload", "makespan_s", "pair_evals_per_s", "step_ms_p50",
                                      "step_ms_p99", "peak_resident", "completed_ok", "saturated",
                                      "latency_vs_alone")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(st, L, flat, args.cpu_sample_pairs)
        v = 2 * cb["pairs"] / (cb["t_bead_s"] + cb["t_nn_s"])
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{cb['pairs']} body pairs of the workload, bead sum and network "
                         f"(FP64, single thread)", "bead_pairs_per_s": cb["bead_pairs_per_s"],
               "nn_pairs_per_s": cb["nn_pairs_per_s"]}
        try:
            cpu["all_cores"] = cpu_baseline_parallel(st, L, flat, args.cpu_sample_pairs,
                                                     os.cpu_count() or 1)
        except Exception as ex:  # reported, not fatal: the single-thread number stands
            cpu["all_cores"] = {"error": repr(ex)}

    clocks = clk.summary()
    path_info = {}
    for p in paths:
        ms = statistics.mean(per_path_ms[p])
        path_info[p] = {"ms_per_md_step": ms, "md_steps_per_s": 1e3 / ms,
                        "pair_evals_per_s": n_pairs[p] / (ms * 1e-3), "pairs": n_pairs[p]}
        if p in path_errors:
            path_info[p]["error"] = path_errors[p]
    if "beads" in path_info:
        for p in paths:
            if p != "beads":
                path_info[p]["speedup_vs_beads"] = path_info["beads"]["ms_per_md_step"] / path_info[p]["ms_per_md_step"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if head == "nn_bf16" else "f32", "data": "synthetic",
            "headline_path": head,
            "headline_model_error": (model_error or {}).get(head),
            "path_dtypes": {"beads": "f32", "nn_fp32": "f32 (SIMT)",
                            "nn_f16x3": "f16 x3 split products, f32 accumulation (FP32 accuracy, "
                                        "parity-tested at the FP32 tolerance)",
                            "nn_bf16": "bf16 products, f32 accumulation"},
            "config": {"workload": f"{N_BODIES} cubes (5x5x5 beads, LJ eps=sigma=1 rc=2.5), "
                                   f"phi={PHI}, NVE dt={DT}; value: MD steps of the {head} path "
                                   f"(each bench step also runs {'+'.join(p for p in paths if p != head)} "
                                   f"on the same state for comparison); MLP 10-{WIDTH}x{DEPTH}-1 SiLU "
                                   f"{'trained on device by force matching on symmetry-reduced configurations' if training else 'random init'}"
                                   + (f"; network pairs closer than {rho_fallback:.3f} sigma (the training set's "
                                      f"smallest contact separation) take the bead sum" if rho_fallback > 0 else ""),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "pair_list": f"Verlet skin {args.skin} sigma, rebuilt on the device when a "
                                    f"centre moves more than skin/2; pairs beyond Rc give exactly zero",
                       "l2": "256 MiB buffer written between steps, outside the per-step events"},
            "paths": path_info, "roofline": roof_nn if head == "nn_bf16" else roof_beads,
            "roofline_beads": roof_beads, "roofline_nn_f16x3": roof_x3,
            "roofline_hbm_step_kernels": {
                k: {"bound": "hbm", "traffic": v["dram_bytes"], "ncu_us": v["ncu_us"],
                    "achieved_gbs": v["dram_bytes"] / (v["ncu_us"] * 1e-6) / 1e9,
                    "peak": pk.get("hbm_gbs", 6800.0),
                    "frac": v["dram_bytes"] / (v["ncu_us"] * 1e-6) / 1e9 / pk.get("hbm_gbs", 6800.0),
                    "source": "ncu dram__bytes and gpu__time_duration (profiles/"
                              "launches_32768_cubes_md_step.md)"}
                for k, v in NCU_STEP_KERNELS.items()},
            "measured_unit_peaks": unit,
            "roofline_nn_fp32": roof_f32, "nn_fp32_simt": simt, "cpu_baseline": cpu,
            "nn_model_error": model_error, "training": training, "serving": serving,
            "nn_bf16_width256": width256, "nve_drift": drift, "training_cylinders_w256": train_cyl,
            "paper_workload_hphc_nvt": paper_wl, "cylinders_per_component_networks": fnet_leg,
            "descriptor_paper6_vs_features10": desc_cmp,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "results_finite": e2e_ok, "path": head,
                    "note": "per step, one rb_step_host_state call: the velocity-Verlet "
                            "state (centres, orientations, momenta, forces) in from one "
                            "page-locked host block, one MD step, the new state and forces out "
                            "to the same block; one host synchronisation per step.  Direct form: "
                            "the step's integrator reads the block from host memory and it and "
                            "the force reduction write the new state back (the bytes cross the "
                            "host link inside the kernels, no copy is queued)",
                    "copies_form": {"value": e2e_value_copies, "unit": UNIT,
                                    "note": "the same with one cudaMemcpyAsync each way around "
                                            "the step"}},
            # per MD step and path: integrate (with the skin check), cell assign,
            # pair build (+ scan), emit (+ finish), pair kernel, reduce; plus the
            # bead fallback kernel on the network paths
            "gpu_launches": args.steps * (6 * len(paths) + (sum(p.startswith("nn") for p in paths)
                                                           if rho_fallback > 0 else 0)),
            "clocks": clocks,
            "peaks_source": how, "wall_s": wall}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
