#!/usr/bin/env python3
"""Benchmark: all-vs-all cRMSD pairs/s (forward + backward) on one B300.

Workload (default): the large combined forward+backward ensemble, N = 8,192 models x L = 500
atoms from 10 seeded natives, sigma ~ U(0.1, 12) A, random rigid motions (33,550,336 pairs).
One step is one pass of the whole hot path over that ensemble:
    pre-pass + all-pairs forward (condensed FP32 matrix, exact-digit BF16 form)
    + one-versus-native scoring of all models (on a second stream)
    + the adjoint of sum_ab w_ab cRMSD_ab (w ~ U[0,1], fixed) to d/dcoords, every pair's
      rotation recomputed from the coordinates (nothing stored by the forward),
as one clusco_crmsd_allpairs_step call (the adjoint's pre-pass beside the forward) plus the
one-versus-native call. ``value`` is pairs per second of that step (P / step time, device time
by CUDA events, inputs resident in HBM). L2 is flushed (a 512 MiB write) before every timed
step, outside the events. ``e2e`` repeats the step through the public API with host buffers:
the step's inputs go host->device from pinned memory and the matrix, the vs-native scores and
the gradient come back device->host inside the timed region.

Extra keys: the forward alone and its ratios to the plain FP32 form and to the exact-integer
CUDA-core form (the accuracy-matched denominator), sampled errors of the matrix and of the
gradient against the FP64 oracle, the rooflines of the two tensor-core kernels, the 50,000 x
1,000 forward, the per-form errors on the precision ensemble, the stored-rotation step and the
5,000 x 300 step (both labelled as departing from the default), and the widened scores (dRMSD,
contact map overlap, GDT_TS / TM-score / MaxSub) on the 5,000 x 300 ensemble.

``--impl reference`` times the FP64 CPU oracle (test infrastructure, the reference arm of
this build) on a bounded sample of the same workload on the host cores.
Under torchrun (N > 1 GPUs) every rank runs an independent replica (the path needs no
exchange); value = pairs of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "all-vs-all cRMSD pairs/s (fwd, fwd+bwd) vs plain FP32, at max err ≤1e-3 Å"
UNIT = "pairs/s"
EPS = 1e-6


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=8192)
    p.add_argument("--L", type=int, default=500)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip every extra measurement (large forward, per-form errors, stored-rotation step, "
                        "5,000 x 300 step, widened scores)")
    p.add_argument("--no-drmsd", action="store_true",
                   help="skip the dRMSD, contact map overlap and GDT / TM-score measurements")
    p.add_argument("--no-large", action="store_true", help="skip the 50,000 x 1,000 forward")
    p.add_argument("--cpu-models", type=int, default=4000, help="models in the oracle's timed sample")
    p.add_argument("--ref-models", type=int, default=600, help="models per step of the reference arm")
    return p.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, device, world):
    """Element-wise maximum of vals over the ranks (each time is the slowest rank's); the values
    themselves at world size 1. The only collective of the replicas: no data crosses ranks."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(units_per_rank, ms, world):
    """Units processed by all ranks per second, timed by the slowest rank."""
    return world * units_per_rank / (ms * 1e-3)


def workload(N, L):
    """The large combined ensemble (10 natives, sigma 0.1-12 A) at N x L, its fixed weights and the
    first native (the vs-native reference)."""
    from paper_1302_4000_b300 import ensembles as E
    e = E.config4(N=N, L=L)
    w = E.weights(N * (N - 1) // 2, 505)
    native = np.ascontiguousarray(e.natives[0].astype(np.float32))
    return e, w, native


def workload_name(N, L):
    return (f"large combined fwd+bwd: N={N} models x L={L} atoms, 10 natives, sigma~U(0.1,12) A, "
            f"{N * (N - 1) // 2} pairs")


class _CtypesNvml:
    """The few NVML calls the clock sampler needs, through ctypes on the driver's libnvidia-ml
    (for hosts where the pynvml module is not importable). Reason bits as in the public nvml.h."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        self._ok(self.lib.nvmlInit_v2(), "nvmlInit_v2")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    @staticmethod
    def _ok(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} returned {rc}")

    def handle(self, uuid, index):
        h = self.ct.c_void_p()
        if uuid and self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), self.ct.byref(h)) == 0:
            return h
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.ct.c_uint(index), self.ct.byref(h)),
                 "nvmlDeviceGetHandleByIndex_v2")
        return h

    def nvmlDeviceGetClockInfo(self, h, kind):
        v = self.ct.c_uint()
        self._ok(self.lib.nvmlDeviceGetClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)), "nvmlDeviceGetClockInfo")
        return v.value

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        v = self.ct.c_uint()
        self._ok(self.lib.nvmlDeviceGetMaxClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)),
                 "nvmlDeviceGetMaxClockInfo")
        return v.value

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.ct.c_ulonglong()
        self._ok(self.reasons_fn(h, self.ct.byref(v)), "clock event reasons")
        return v.value


class Clocks:
    """SM clock and clock-event reasons sampled through NVML every ~10 ms in a thread, so that a
    timed region of a fraction of a second still carries samples; window() keeps those taken
    between two perf_counter() stamps. NVML through the pynvml module, else through ctypes on
    the driver's library. Reading only: no setting of the GPU is changed."""

    NAMES = (("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
             ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
             ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
             ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"))

    def __init__(self, gpu_index, uuid=None, period=0.01):
        self.samples = []
        self.smax, self.source = None, None
        self.period = period
        self.stop_ev = threading.Event()
        self.err = None
        self.nv = None
        errs = []
        try:
            import pynvml
            pynvml.nvmlInit()
            h = None
            if uuid:
                try:
                    h = pynvml.nvmlDeviceGetHandleByUUID(uuid)
                except Exception:
                    h = None
            self.h = h if h is not None else pynvml.nvmlDeviceGetHandleByIndex(gpu_index)
            self.smax = float(pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM))
            self.nv, self.source = pynvml, "NVML (pynvml)"
        except Exception as ex:
            errs.append(f"pynvml: {ex}")
        if self.nv is None:
            try:
                nv = _CtypesNvml()
                self.h = nv.handle(uuid, gpu_index)
                self.smax = float(nv.nvmlDeviceGetMaxClockInfo(self.h, nv.NVML_CLOCK_SM))
                self.nv, self.source = nv, "NVML (ctypes on libnvidia-ml.so.1)"
            except Exception as ex:
                errs.append(f"ctypes NVML: {ex}")
        self.smi = None
        if self.nv is None:  # no NVML: nvidia-smi's own sampling loop, else the line says so
            self.err = "NVML unavailable: " + "; ".join(errs)
            import shutil
            if shutil.which("nvidia-smi"):
                self.smi_index = gpu_index if uuid is None else uuid
        self.th = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        nv = self.nv
        while not self.stop_ev.is_set():
            try:
                t = time.perf_counter()
                sm = float(nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM))
                r = int(nv.nvmlDeviceGetCurrentClocksEventReasons(self.h))
                self.samples.append((t, sm, r))
            except Exception as ex:
                self.err = str(ex)
                return
            time.sleep(self.period)

    SMI_FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                  "clocks_event_reasons.sw_power_cap")

    def start(self):
        if self.nv is not None:
            self.th.start()
        elif hasattr(self, "smi_index"):
            import subprocess
            import tempfile
            self.smi_file = tempfile.TemporaryFile(mode="w+")
            self.wall_minus_perf = time.time() - time.perf_counter()
            self.smi = subprocess.Popen(["nvidia-smi", "-i", str(self.smi_index), "--query-gpu=" + self.SMI_FIELDS,
                                         "--format=csv,noheader,nounits", "-lms", "100"],
                                        stdout=self.smi_file, stderr=subprocess.DEVNULL)

    def _smi_collect(self):
        """Ends this sampler's own nvidia-smi child and converts its rows (wall-clock stamps) into
        perf_counter samples."""
        import datetime
        if self.smi is not None:
            self.smi.terminate()
            try:
                self.smi.wait(timeout=5)
            except Exception:
                self.smi.kill()
            self.smi = None
            self.smi_file.seek(0)
            bits = (8, 64, 32, 4)  # the NVML reason bits of the four fields, in NAMES order below
            for row in self.smi_file.read().splitlines():
                f = [x.strip() for x in row.split(",")]
                if len(f) != 7:
                    continue
                try:
                    wall = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    sm, smax = float(f[1]), float(f[2])
                except ValueError:
                    continue
                r = 0
                for b, v in zip(bits, f[3:]):
                    if v.lower() == "active":
                        r |= b
                self.samples.append((wall - self.wall_minus_perf, sm, r))
                self.smax = smax
            self.smi_file.close()
            self.source = "nvidia-smi -lms 100 (NVML not importable)"

    def stop(self):
        self.stop_ev.set()
        if self.th.is_alive():
            self.th.join(timeout=2)
        self._smi_collect()

    def window(self, t0, t1):
        if self.nv is None and self.smi is not None:
            self._smi_collect()
            self.nv = _CtypesNvml  # reason bit constants only
        if self.nv is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [self.err], "samples": 0}
        sel = [s for s in self.samples if t0 <= s[0] <= t1]
        reasons = set()
        for _, _, r in sel:
            for nm, const in self.NAMES:
                if r & getattr(self.nv, const):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(s[1] for s in sel) if sel else None, "sm_max_mhz": self.smax,
                "reasons": sorted(reasons), "samples": len(sel),
                "source": f"{self.source}, every ~10 ms, timed region only"}


def csrc_hash():
    """sha256 over every source file of the library (names and contents, sorted by name): a
    kernel's counters stand only for the sources they were taken from, headers included."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1302_4000_b300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def counter_for(fname, key, N, L):
    """A per-launch counter of a kernel (DRAM bytes in traffic.txt, warp instructions in
    issue.txt) from its committed ncu summary, or None for another workload than the one captured
    (N models of L atoms) or once any library source has changed since the counters were taken
    (csrc_hash recorded beside them)."""
    try:
        h = csrc_hash()
        for line in open(os.path.join(ROOT, "profiles", fname)):
            parts = line.split()
            if (len(parts) == 6 and parts[0] == key and parts[1] == h and int(parts[2]) == N
                    and int(parts[3]) == L):
                return float(parts[4])
    except (OSError, ValueError):
        pass
    return None


def traffic_for(key, N, L):
    return counter_for("traffic.txt", key, N, L)


def issue_for(key, N, L):
    return counter_for("issue.txt", key, N, L)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, 1400.0, "fallback"


def roofline(kernel, launch_ms, timing, flop, hbm_bytes, key, N, L, sm_mhz, n_sms=148):
    """The two-term roofline of one kernel launch: its algorithmic flop at the measured bf16 peak
    against its algorithmic bytes at the measured HBM bandwidth; the larger term bounds the kernel,
    and frac = that term's time / the launch's time (= achieved / peak in the bound's unit). The
    third term is the issue bound: the launch's warp instructions (ncu) at one per scheduler and
    cycle on every SM; frac_3term divides the largest of the three terms by the launch time."""
    hbm, bf16, _, kind = peaks()
    t_tensor = flop / (bf16 * 1e12)
    t_hbm = hbm_bytes / (hbm * 1e9)
    s = launch_ms * 1e-3
    if t_tensor >= t_hbm:
        r = {"bound": "tensor", "achieved": flop / s / 1e12, "peak": bf16, "unit": "TFLOP/s",
             "peak_kind": f"{kind} bf16 burst"}
    else:
        r = {"bound": "hbm", "achieved": hbm_bytes / s / 1e9, "peak": hbm, "unit": "GB/s",
             "peak_kind": f"{kind} HBM copy"}
    r["frac"] = r["achieved"] / r["peak"]
    r.update({"kernel": kernel, "launch_ms": launch_ms, "timing": timing, "algorithmic_flop": flop,
              "algorithmic_bytes": hbm_bytes, "t_tensor_ms": t_tensor * 1e3, "t_hbm_ms": t_hbm * 1e3,
              "traffic": traffic_for(key, N, L)})
    inst = issue_for(key, N, L)
    if inst is not None and sm_mhz:
        t_issue = inst / (4 * n_sms * sm_mhz * 1e6)
        r["issue_3term"] = {"warp_instructions": inst, "t_issue_ms": t_issue * 1e3, "clock_mhz": sm_mhz,
                            "frac_3term": max(t_tensor, t_hbm, t_issue) / s}
    else:
        r["issue_3term"] = None
    return r


def cpu_baseline(e, w, native, n_models):
    """The FP64 oracle as it stands, on all pairs among the first n_models models."""
    import oracle
    X = np.ascontiguousarray(e.coords[:n_models])
    n = X.shape[0]
    from paper_1302_4000_b300 import ensembles as E
    ws = E.weights(n * (n - 1) // 2, 7).astype(np.float64)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.crmsd_allpairs(X)
    oracle.crmsd_vs_ref(X, native)
    oracle.crmsd_grad(X, ws, EPS)
    dt = time.perf_counter() - t0
    P = n * (n - 1) // 2
    return {"value": P / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {P} pairs among the first {n} models of the {e.N} x {e.L} ensemble "
                      f"(fwd + vs-native + gradient), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    e, w, native = workload(args.N, args.L)
    import oracle
    oracle.load()
    times = []
    n = args.ref_models
    for it in range(args.warmup + args.steps):
        r = cpu_baseline(e, w, native, n)
        if it >= args.warmup:
            times.append(r)
    v = statistics.mean(t["value"] for t in times)
    P = n * (n - 1) // 2
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * P / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.N, args.L) + f" (bounded sample: {n} models per step)",
                       "l2": "n/a (CPU)"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": times[0]["cores"], "kind": "oracle",
                             "sample": times[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Timer:
    """K timed repetitions of fn on the current stream after W untimed ones, each bracketed by CUDA
    events, with a 512 MiB write before each (outside the events) so that L2 starts cold."""

    def __init__(self, torch, flush, world, dist):
        self.torch, self.flush, self.world, self.dist = torch, flush, world, dist

    def __call__(self, fn, k, w, prof=False, split=False):
        torch = self.torch
        stream = torch.cuda.current_stream()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k)]
        for _ in range(w):
            if split:
                fn(ev[0])
            else:
                fn()
        torch.cuda.synchronize()
        if self.world > 1:
            self.dist.barrier()
        torch.cuda.synchronize()
        if prof:  # the library brackets each tensor-core kernel launch with events on its stream
            from paper_1302_4000_b300 import clusco
            clusco.profile_enable(True)
        t0 = time.perf_counter()
        for e4 in ev:
            self.flush.fill_(1)
            if split:
                fn(e4)
            else:
                e4[0].record(stream)
                fn()
                e4[3].record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if prof:
            from paper_1302_4000_b300 import clusco
            clusco.profile_enable(False)
        if self.world > 1:
            self.dist.barrier()
        tot = [e4[0].elapsed_time(e4[3]) for e4 in ev]
        out = {"ms": tot, "t0": t0, "t1": t1}
        if split:
            out["a"] = [e4[0].elapsed_time(e4[1]) for e4 in ev]
            out["b"] = [e4[2].elapsed_time(e4[3]) for e4 in ev]
        return out


def sampled_pairs(N, n, seed):
    rng = np.random.default_rng(seed)
    ia = rng.integers(0, N, 4 * n)
    ib = rng.integers(0, N, 4 * n)
    keep = ia != ib
    ia, ib = np.minimum(ia[keep], ib[keep])[:n], np.maximum(ia[keep], ib[keep])[:n]
    return ia, ib, ia * N - ia * (ia + 1) // 2 + (ib - ia - 1)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1302_4000_b300 import build, clusco

    build.build()  # no-op unless a library source is newer than the built library
    ws_, rank, local = dist_env()
    if ws_ > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = clusco.load()
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        uuid = None
    clocks = Clocks(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0, uuid)
    clocks.start()
    form = clusco.FORM_BF16_EXACT2

    e, w, native = workload(args.N, args.L)
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    X = torch.from_numpy(e.coords).to(dev)
    W = torch.from_numpy(w).to(dev)
    ref = torch.from_numpy(native).to(dev)
    out = torch.empty(P, dtype=torch.float32, device=dev)
    vs = torch.empty(N, dtype=torch.float32, device=dev)
    grad = torch.empty_like(X)
    ws_step = torch.empty(clusco.workspace_bytes(clusco.OP_STEP, N, L, form), dtype=torch.uint8, device=dev)
    ws_vs = torch.empty(clusco.workspace_bytes(clusco.OP_VS_REF, N, L, form), dtype=torch.uint8, device=dev)
    ws_all = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N, L, form), dtype=torch.uint8, device=dev)
    ws_bw = torch.empty(clusco.workspace_bytes(clusco.OP_BACKWARD, N, L, form), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    timer = Timer(torch, flush, ws_, dist)

    # one-versus-native needs neither the forward nor the adjoint: it runs on a second stream,
    # forked at the start of the step and joined before its end
    side = torch.cuda.Stream()
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def vs_native(st):
        clusco.crmsd_vs_ref(X, ref, out=vs, workspace=ws_vs, stream=st)

    def step():
        fork.record(stream)
        side.wait_event(fork)
        vs_native(side)
        join.record(side)
        clusco.crmsd_allpairs_step(X, W, form, EPS, out=out, grad_coords=grad, workspace=ws_step)
        stream.wait_event(join)

    def step_split(evs):
        # the forward and the adjoint as two calls, with events between them (the breakdown)
        evs[0].record(stream)
        clusco.crmsd_allpairs(X, form, out=out, workspace=ws_all)
        evs[1].record(stream)
        evs[2].record(stream)
        clusco.crmsd_allpairs_backward(X, W, out, EPS, form, grad_coords=grad, workspace=ws_bw)
        evs[3].record(stream)

    # kernels of this library per step: forward (pre-pass, pairs, refinement of flagged pairs),
    # one-versus-native (reference pre-pass, scores), adjoint (pre-pass, FP16 split, max |w|,
    # sweep, reduction, near-duplicate pass)
    launches_per_step = 3 + 2 + 6

    main = timer(step, args.steps, args.warmup, prof=True)
    clk = clocks.window(main["t0"], main["t1"])
    kern = {}
    for name, kid in (("pairs", clusco.KERNEL_PAIRS), ("adjoint", clusco.KERNEL_ADJOINT)):
        tot_ms, n = clusco.profile_read(kid)
        kern[name] = (tot_ms / n) if n else None
    if clusco.sync_status() != 0:
        raise RuntimeError("device status set during the timed steps: " + lib.clusco_last_error().decode())
    sp = timer(step_split, max(3, args.steps // 4), 2, split=True)
    ms = statistics.mean(main["ms"])
    fms, bms = statistics.mean(sp["a"]), statistics.mean(sp["b"])
    ms, fms, bms = max_over_ranks([ms, fms, bms], dev, ws_)

    # plain-form forward for the "vs plain FP32" ratio (same GPU, same inputs)
    ws_p = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                       device=dev)
    out_p = torch.empty_like(out)
    plain_fwd = statistics.mean(timer(lambda: clusco.crmsd_allpairs(X, clusco.FORM_FP32_SIMT, out=out_p,
                                                                     workspace=ws_p), 3, 1)["ms"])
    plain_fwd = max_over_ranks([plain_fwd], dev, ws_)[0]
    del ws_p
    # the accuracy-matched CUDA-core denominator: the exact-integer form (24-bit fixed point,
    # int64 sums, FP64 refinement below its FP32 bound), same inputs
    ws_p = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N, L, clusco.FORM_INT_SIMT), dtype=torch.uint8,
                       device=dev)
    int_fwd = statistics.mean(timer(lambda: clusco.crmsd_allpairs(X, clusco.FORM_INT_SIMT, out=out_p,
                                                                   workspace=ws_p), 3, 1)["ms"])
    int_fwd = max_over_ranks([int_fwd], dev, ws_)[0]
    if clusco.sync_status() != 0:
        raise RuntimeError("device status set during the exact-integer forward: " + lib.clusco_last_error().decode())
    del ws_p, out_p

    # accuracy of this run's outputs against the oracle (outside timing): sampled pairs of the
    # matrix, sampled rows of the gradient
    acc = None
    if rank == 0:
        import oracle
        clusco.crmsd_allpairs_step(X, W, form, EPS, out=out, grad_coords=grad, workspace=ws_step)
        torch.cuda.synchronize()
        ia, ib, idx = sampled_pairs(N, 4000, 3)
        got = out.cpu().numpy()[idx].astype(np.float64)
        c_err = float(np.abs(got - oracle.crmsd_pairs(e.coords, ia, ib)).max())
        rows = np.array([0, 1, N // 2, N - 1])
        gref = oracle.crmsd_grad_rows(e.coords, w.astype(np.float64), rows, EPS)
        gg = grad[torch.from_numpy(rows).to(dev)].double().cpu().numpy()
        rel = (np.linalg.norm((gg - gref).reshape(len(rows), -1), axis=1)
               / np.linalg.norm(gref.reshape(len(rows), -1), axis=1))
        vs_err = float(np.abs(vs.double().cpu().numpy() - oracle.crmsd_vs_ref(e.coords, native)).max())
        acc = {"max_err_sampled_A": c_err, "pairs_sampled": int(len(idx)), "vs_native_max_err_A": vs_err,
               "grad_max_rel_err_rows": float(rel.max()), "grad_rows": rows.tolist(),
               "tolerances": "matrix 1e-3 A (split-BF16); gradient 1e-3 relative per model"}

    # e2e through the public API with host buffers. Each step copies its inputs (coords,
    # weights, native) host -> device from pinned memory and its results (matrix, vs-native
    # scores, gradient) back, all inside the timed region. Steps are pipelined the way a user
    # streaming ensembles would run them: three device buffer sets, the uploads of step k+1 and
    # the downloads of step k-1 on their own streams overlap the compute of step k. Throughput =
    # steps / (first upload start .. last download end). The working set is larger than L2, so no
    # flush between steps.
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(e.coords).pin_memory()
        Wh = torch.from_numpy(w).pin_memory()
        Rh = torch.from_numpy(native).pin_memory()
        out_h = torch.empty(P, dtype=torch.float32).pin_memory()
        vs_h = torch.empty(N, dtype=torch.float32).pin_memory()
        g_h = torch.empty(X.shape, dtype=torch.float32).pin_memory()
        nbuf = 3
        bufs = []
        for _ in range(nbuf):
            bufs.append({"X": torch.empty_like(X), "W": torch.empty_like(W), "R": torch.empty_like(ref),
                         "out": torch.empty_like(out), "vs": torch.empty_like(vs), "g": torch.empty_like(grad),
                         "in_ready": torch.cuda.Event(), "done": torch.cuda.Event(), "copied": torch.cuda.Event(),
                         "vs_done": torch.cuda.Event()})
        s_in, s_cmp, s_out, s_vs = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_run(nsteps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(s_in)
            for k in range(nsteps):
                b = bufs[k % nbuf]
                with torch.cuda.stream(s_in):
                    if k >= nbuf:  # this buffer set's previous results are on the host
                        s_in.wait_event(b["copied"])
                    b["X"].copy_(Xh, non_blocking=True)
                    b["W"].copy_(Wh, non_blocking=True)
                    b["R"].copy_(Rh, non_blocking=True)
                    b["in_ready"].record(s_in)
                s_cmp.wait_event(b["in_ready"])
                s_vs.wait_event(b["in_ready"])
                clusco.crmsd_vs_ref(b["X"], b["R"], out=b["vs"], workspace=ws_vs, stream=s_vs)
                b["vs_done"].record(s_vs)
                clusco.crmsd_allpairs_step(b["X"], b["W"], form, EPS, out=b["out"], grad_coords=b["g"],
                                           workspace=ws_step, stream=s_cmp)
                s_cmp.wait_event(b["vs_done"])
                b["done"].record(s_cmp)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(b["done"])
                    out_h.copy_(b["out"], non_blocking=True)
                    vs_h.copy_(b["vs"], non_blocking=True)
                    g_h.copy_(b["g"], non_blocking=True)
                    b["copied"].record(s_out)
            ev1.record(s_out)
            torch.cuda.synchronize()
            return ev0.elapsed_time(ev1)

        e2e_run(max(args.warmup, nbuf))
        if ws_ > 1:
            dist.barrier()
        e_ms = e2e_run(args.steps) / args.steps
        e_ms = max_over_ranks([e_ms], dev, ws_)[0]
        h2d = Xh.numel() * 4 + Wh.numel() * 4 + Rh.numel() * 4
        d2h = out_h.numel() * 4 + vs_h.numel() * 4 + g_h.numel() * 4
        # the host link's own rates with the same pinned buffers (the weights up, the matrix down):
        # one direction at a time, then both at once, as the pipelined steps run them
        b0 = bufs[0]

        def link_gbs(pairs, nrep=5):
            for st, fn in pairs:
                with torch.cuda.stream(st):
                    fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(nrep):
                for st, fn in pairs:
                    with torch.cuda.stream(st):
                        fn()
            torch.cuda.synchronize()
            return nrep * Wh.numel() * 4 / (time.perf_counter() - t0) / 1e9
        up = lambda: b0["W"].copy_(Wh, non_blocking=True)
        down = lambda: out_h.copy_(b0["out"], non_blocking=True)
        l_up = link_gbs([(s_in, up)])
        l_down = link_gbs([(s_out, down)])
        l_both = link_gbs([(s_in, up), (s_out, down)])
        e2e = {"value": whole_job_rate(P, e_ms, ws_), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e_ms,
               "pipelined": "three buffer sets; uploads of step k+1 and downloads of step k-1 overlap step k",
               "calls": "clusco_crmsd_allpairs_step and clusco_crmsd_vs_ref per step",
               "l2": "working set larger than L2, no flush",
               "link_GBs": {"h2d": l_up, "d2h": l_down, "each_way_when_both": l_both,
                            "floor_ms_per_step": max(h2d, d2h) / (l_both * 1e6)}}
        del bufs

    # rooflines of the two tensor-core kernels (per launch, one launch each per step). Forward:
    # 18 L flop per pair (the 3 x 3 covariance over L atoms) against the 4-byte condensed output.
    # Adjoint: the second contraction, 2 (3N)^2 L flop, against its algorithmic bytes (the matrix
    # and the weights read, 8 bytes per pair, the coordinates read and the gradient written,
    # 24 L bytes per model).
    sm_mhz = clk.get("sm_mhz")
    r_fwd = roofline("pairs_tc_kernel<EXACT2> (forward, exact-digit BF16 covariance + eq. 2 epilogue)",
                     kern["pairs"] or fms, "kernel launch events" if kern["pairs"] else "API call bracket",
                     18.0 * L * P, 4.0 * P, "pairs_tc", N, L, sm_mhz)
    r_bwd = roofline("bwd_rc_kernel (adjoint, rotations recomputed; second contraction 2 (3N)^2 L)",
                     kern["adjoint"] or bms, "kernel launch events" if kern["adjoint"] else "API call bracket",
                     2.0 * (3 * N) ** 2 * L, 8.0 * P + 24.0 * N * L, "bwd_rc", N, L, sm_mhz)
    dominant, other = (r_bwd, r_fwd) if r_bwd["launch_ms"] >= r_fwd["launch_ms"] else (r_fwd, r_bwd)

    line = {"metric": METRIC, "value": whole_job_rate(P, ms, ws_), "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16(exact int)+f32/f64 fwd; f16x3+f32 bwd",
            "data": "synthetic",
            "config": {"workload": workload_name(N, L), "form": "bf16_exact2", "pairs": P,
                       "step": "one clusco_crmsd_allpairs_step call (forward, then the adjoint with its pre-pass "
                               "beside the forward) + clusco_crmsd_vs_ref of all models against the first native "
                               "on a second stream",
                       "adjoint": "recomputed: every pair's covariance and rotation recomputed from the coordinates, "
                                  "nothing stored by the forward",
                       "l2": "flushed (512 MiB write) before each timed step", "parallelism": f"replicas x{ws_}"},
            "fwd": {"value": whole_job_rate(P, fms, ws_), "unit": UNIT, "ms": fms},
            "bwd": {"value": whole_job_rate(P, bms, ws_), "unit": UNIT, "ms": bms},
            "vs_plain_fp32_fwd": plain_fwd / fms, "plain_fp32_fwd_ms": plain_fwd,
            "vs_plain_exact_int": int_fwd / fms, "plain_exact_int_fwd_ms": int_fwd,
            "accuracy": acc,
            "roofline": dominant, "roofline_other": other,
            "clocks": clk, "gpu_launches": launches_per_step * args.steps}
    if e2e:
        line["e2e"] = e2e
    if not args.no_extra:
        extra(args, line, torch, clusco, lib, dev, timer, ws_, rank, dist)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(e, w, native, args.cpu_models)
    clocks.stop()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        dist.destroy_process_group()


def extra(args, line, torch, clusco, lib, dev, timer, ws_, rank, dist):
    """Measurements beside the headline step, each under its own key."""
    from paper_1302_4000_b300 import ensembles as E
    form = clusco.FORM_BF16_EXACT2

    def status(what):
        if clusco.sync_status() != 0:
            raise RuntimeError(f"device status set during {what}: " + lib.clusco_last_error().decode())

    # ---- the large forward: 50,000 x 1,000 (1.25e9 pairs, 5 GB condensed output kept on device;
    # the device -> host copy of the matrix timed separately)
    if not args.no_large:
        e4 = E.config4()
        N4, L4 = e4.N, e4.L
        P4 = N4 * (N4 - 1) // 2
        X4 = torch.from_numpy(e4.coords).to(dev)
        out4 = torch.empty(P4, dtype=torch.float32, device=dev)
        ws4 = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N4, L4, form), dtype=torch.uint8, device=dev)
        r4 = timer(lambda: clusco.crmsd_allpairs(X4, form, out=out4, workspace=ws4), 3, 1, prof=True)
        k4, n4 = clusco.profile_read(clusco.KERNEL_PAIRS)
        status("the 50,000 x 1,000 forward")
        f4 = max_over_ranks([statistics.mean(r4["ms"])], dev, ws_)[0]
        host4 = torch.empty(P4, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host4.copy_(out4)
        d2h_s = time.perf_counter() - t0
        err4 = None
        if rank == 0:
            import oracle
            ia, ib, idx = sampled_pairs(N4, 2000, 44)
            err4 = float(np.abs(host4.numpy()[idx].astype(np.float64) - oracle.crmsd_pairs(e4.coords, ia, ib)).max())
        line["large_fwd"] = {
            "workload": f"large combined forward: N={N4} models x L={L4} atoms, 10 natives, sigma~U(0.1,12) A",
            "pairs": P4, "value": whole_job_rate(P4, f4, ws_), "unit": UNIT, "ms": f4,
            "kernel_launch_ms": (k4 / n4) if n4 else None,
            "roofline": roofline("pairs_tc_kernel<EXACT2> (forward)", (k4 / n4) if n4 else f4,
                                 "kernel launch events" if n4 else "API call bracket", 18.0 * L4 * P4, 4.0 * P4,
                                 "pairs_tc", N4, L4, line["clocks"].get("sm_mhz")),
            "output_GB": P4 * 4 / 1e9, "output": "one call, condensed matrix kept on device",
            "d2h_ms": d2h_s * 1e3, "d2h_GBs": P4 * 4 / d2h_s / 1e9, "max_err_sampled_A": err4}
        del X4, out4, ws4, host4, e4
        torch.cuda.empty_cache()

    # ---- per-form errors on the precision ensemble (20,000 x 150: half the models in near-duplicate
    # clusters, sigma 0.02-0.5 A around their centres): max and p99 |d cRMSD| against the FP64 oracle
    # over every intra-cluster pair and 20,000 random pairs, per form, with each form's forward time
    if rank == 0:
        import oracle
        e2 = E.config2()
        N2 = e2.N
        X2 = torch.from_numpy(e2.coords).to(dev)
        cl = e2.extra["cluster"]
        ia_l, ib_l = [], []
        for c in np.unique(cl[cl >= 0]):
            m = np.flatnonzero(cl == c)
            a, b = np.triu_indices(len(m), 1)
            ia_l.append(m[a])
            ib_l.append(m[b])
        na, nb = np.concatenate(ia_l), np.concatenate(ib_l)
        na, nb = np.minimum(na, nb), np.maximum(na, nb)
        ra, rb, _ = sampled_pairs(N2, 20000, 22)
        ref_nd = oracle.crmsd_pairs(e2.coords, na, nb)
        ref_rd = oracle.crmsd_pairs(e2.coords, ra, rb)
        idx_nd = torch.from_numpy(na * N2 - na * (na + 1) // 2 + (nb - na - 1)).to(dev)
        idx_rd = torch.from_numpy(ra * N2 - ra * (ra + 1) // 2 + (rb - ra - 1)).to(dev)
        pf = {"workload": f"precision ensemble N={N2} x L={e2.L}: {len(na)} intra-cluster (near-duplicate) pairs, "
                          f"c from {ref_nd.min():.3f} to {ref_nd.max():.2f} A, and {len(ra)} random pairs"}
        out2 = torch.empty(N2 * (N2 - 1) // 2, dtype=torch.float32, device=dev)
        for name, f in (("bf16_exact2", clusco.FORM_BF16_EXACT2), ("bf16x3", clusco.FORM_BF16X3),
                        ("tf32", clusco.FORM_TF32), ("fp32_simt", clusco.FORM_FP32_SIMT),
                        ("int_simt", clusco.FORM_INT_SIMT)):
            ws2 = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N2, e2.L, f), dtype=torch.uint8, device=dev)
            t = timer(lambda: clusco.crmsd_allpairs(X2, f, out=out2, workspace=ws2), 2, 1)
            status(f"the precision forward ({name})")
            d_nd = np.abs(out2[idx_nd].double().cpu().numpy() - ref_nd)
            d_rd = np.abs(out2[idx_rd].double().cpu().numpy() - ref_rd)
            pf[name] = {"near_dup_max": float(d_nd.max()), "near_dup_p99": float(np.quantile(d_nd, 0.99)),
                        "random_max": float(d_rd.max()), "random_p99": float(np.quantile(d_rd, 0.99)),
                        "fwd_ms": statistics.mean(t["ms"]),
                        "meets_1e-3_A": bool(max(d_nd.max(), d_rd.max()) <= 1e-3),
                        "meets_1e-4_A": bool(max(d_nd.max(), d_rd.max()) <= 1e-4)}
            del ws2
        line["per_form_error"] = pf
        del X2, out2
        torch.cuda.empty_cache()

    # ---- the stored-rotation step (departs from the default: the forward stores every pair's
    # rotation, 48 bytes per pair, and the adjoint contracts from them) on the default ensemble
    N, L = args.N, args.L
    if L <= 512:
        e, w, native = workload(N, L)
        P = N * (N - 1) // 2
        X = torch.from_numpy(e.coords).to(dev)
        W = torch.from_numpy(w).to(dev)
        out = torch.empty(P, dtype=torch.float32, device=dev)
        grad = torch.empty_like(X)
        rot = torch.empty((P, clusco.ROT_STRIDE), dtype=torch.float32, device=dev)
        wsr = torch.empty(clusco.workspace_bytes(clusco.OP_STEP_ROT, N, L, form), dtype=torch.uint8, device=dev)
        t = timer(lambda: clusco.crmsd_allpairs_step_rot(X, W, form, EPS, out=out, rot=rot, grad_coords=grad,
                                                         workspace=wsr), 5, 2)
        status("the stored-rotation step")
        m = max_over_ranks([statistics.mean(t["ms"])], dev, ws_)[0]
        line["stored_rotations_step"] = {
            "departs_from_default": "the forward stores each pair's rotation (48 B/pair, "
                                    f"{P * 48 / 1e9:.2f} GB here); the default recomputes them",
            "value": whole_job_rate(P, m, ws_), "unit": UNIT, "ms": m, "step": "clusco_crmsd_allpairs_step_rot "
            "(no vs-native)"}
        del X, W, out, grad, rot, wsr
        torch.cuda.empty_cache()

    # ---- the 5,000 x 300 decoy ensemble (5 natives, sigma 0.5-10 A): the recomputing step there,
    # and the widened scores
    e1 = E.config1()
    N1, L1 = e1.N, e1.L
    P1 = N1 * (N1 - 1) // 2
    X1 = torch.from_numpy(e1.coords).to(dev)
    W1 = torch.from_numpy(E.weights(P1, E.SEED_BASE + 101)).to(dev)
    out1 = torch.empty(P1, dtype=torch.float32, device=dev)
    g1 = torch.empty_like(X1)
    ws1 = torch.empty(clusco.workspace_bytes(clusco.OP_STEP, N1, L1, form), dtype=torch.uint8, device=dev)
    t = timer(lambda: clusco.crmsd_allpairs_step(X1, W1, form, EPS, out=out1, grad_coords=g1, workspace=ws1), 10, 3)
    status("the 5,000 x 300 step")
    m = max_over_ranks([statistics.mean(t["ms"])], dev, ws_)[0]
    line["step_5000x300"] = {"workload": f"decoy ensemble N={N1} x L={L1}, 5 natives, sigma~U(0.5,10) A",
                             "value": whole_job_rate(P1, m, ws_), "unit": UNIT, "ms": m,
                             "step": "clusco_crmsd_allpairs_step (no vs-native)"}
    del out1, g1, ws1, W1
    if not args.no_drmsd:
        widened(line, torch, clusco, dev, timer, ws_, rank, e1, X1, status)
    del X1
    torch.cuda.empty_cache()


def widened(line, torch, clusco, dev, timer, ws_, rank, e, X, status):
    """All-versus-all dRMSD (eq. 5), contact map overlap (eq. 6, eq. 7) and GDT_TS / TM-score /
    MaxSub against a reference (eq. 3, eq. 4) on the 5,000 x 300 ensemble."""
    hbm, bf16, _, pk_kind = peaks()
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    K = L * (L - 1) // 2
    wl = f"decoy ensemble N={N} x L={L}"
    # dRMSD: the exact Gram of the 16-bit rounded distances (2 K flop per pair over the K atom
    # pairs, executed as four BF16 digit-product classes) against the plain FP32 form
    ws_d = torch.empty(clusco.workspace_bytes(clusco.OP_DRMSD, N, L, clusco.FORM_BF16_EXACT2), dtype=torch.uint8,
                       device=dev)
    out_d = torch.empty(P, dtype=torch.float32, device=dev)
    d = timer(lambda: clusco.drmsd_allpairs(X, clusco.FORM_BF16_EXACT2, out=out_d, workspace=ws_d), 5, 2, prof=True)
    tot_ms, n = clusco.profile_read(clusco.KERNEL_DRMSD)
    dk_ms = tot_ms / n if n else None
    ws_dp = torch.empty(clusco.workspace_bytes(clusco.OP_DRMSD, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                        device=dev)
    out_dp = torch.empty_like(out_d)
    dp = timer(lambda: clusco.drmsd_allpairs(X, clusco.FORM_FP32_SIMT, out=out_dp, workspace=ws_dp), 2, 1)
    status("the dRMSD calls")
    d_ms, dp_ms = max_over_ranks([statistics.mean(d["ms"]), statistics.mean(dp["ms"])], dev, ws_)
    d_err = None
    if rank == 0:
        import oracle
        ia, ib, idx = sampled_pairs(N, 4000, 4)
        d_err = float(np.abs(out_d.cpu().numpy()[idx].astype(np.float64) - oracle.drmsd_pairs(e.coords, ia, ib)).max())
    kms = dk_ms if dk_ms else d_ms
    ach = 2.0 * K * P / (kms * 1e-3) / 1e12
    line["drmsd"] = {"workload": wl, "value": whole_job_rate(P, d_ms, ws_), "unit": UNIT, "ms": d_ms,
                     "form": "bf16_exact2", "vs_plain_fp32": dp_ms / d_ms, "plain_fp32_ms": dp_ms,
                     "max_err_sampled_A": d_err,
                     "roofline": {"kernel": "drmsd_tc_kernel (Gram of the rounded distances, 2 K flop/pair)",
                                  "launch_ms": kms, "timing": "kernel launch events" if dk_ms else "API call bracket",
                                  "bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                                  "frac": ach / bf16, "peak_kind": f"{pk_kind} bf16 burst",
                                  "traffic": traffic_for("drmsd_tc", N, L)}}
    del ws_d, out_d, ws_dp, out_dp
    # contact map overlap at an 8 A cutoff: E4M3 0/1 maps on kind::f8f6f4 (its peak is the FP8
    # rate, twice the measured BF16) against the plain bit-count form
    ws_c = torch.empty(clusco.workspace_bytes(clusco.OP_CMO, N, L, clusco.FORM_FP8_EXACT), dtype=torch.uint8,
                       device=dev)
    out_c = torch.empty(P, dtype=torch.float32, device=dev)
    c = timer(lambda: clusco.cmo_allpairs(X, 8.0, clusco.FORM_FP8_EXACT, out=out_c, workspace=ws_c), 5, 2, prof=True)
    tot_ms, n = clusco.profile_read(clusco.KERNEL_CMO)
    ck_ms = tot_ms / n if n else None
    ws_cp = torch.empty(clusco.workspace_bytes(clusco.OP_CMO, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                        device=dev)
    out_cp = torch.empty_like(out_c)
    cp = timer(lambda: clusco.cmo_allpairs(X, 8.0, clusco.FORM_FP32_SIMT, out=out_cp, workspace=ws_cp), 3, 1)
    status("the contact-map calls")
    c_ms, cp_ms = max_over_ranks([statistics.mean(c["ms"]), statistics.mean(cp["ms"])], dev, ws_)
    c_err = None
    if rank == 0:
        import oracle
        ia, ib, idx = sampled_pairs(N, 4000, 6)
        c_err = float(np.abs(out_c.cpu().numpy()[idx].astype(np.float64)
                             - oracle.cmo_pairs(e.coords, ia, ib, 8.0)).max())
    kms = ck_ms if ck_ms else c_ms
    ach = 2.0 * K * P / (kms * 1e-3) / 1e12
    line["cmo"] = {"workload": wl, "value": whole_job_rate(P, c_ms, ws_), "unit": UNIT, "ms": c_ms,
                   "form": "fp8_exact", "cutoff_A": 8.0, "vs_plain_popcount": cp_ms / c_ms,
                   "plain_popcount_ms": cp_ms, "max_err_sampled_pct": c_err,
                   "roofline": {"kernel": "cmo_tc_kernel (Gram of the 0/1 contact maps, 2 K flop/pair)",
                                "launch_ms": kms, "timing": "kernel launch events" if ck_ms else "API call bracket",
                                "bound": "tensor", "achieved": ach, "peak": 2.0 * bf16, "unit": "TFLOP/s",
                                "frac": ach / (2.0 * bf16), "peak_kind": f"{pk_kind} bf16 burst x 2 (FP8 nominal ratio)",
                                "traffic": traffic_for("cmo_tc", N, L)}}
    del ws_c, out_c, ws_cp, out_cp
    # GDT_TS / TM-score / MaxSub of every model against the first native, with the oracle timed on
    # a bounded sample of models on the host cores
    if 3 <= L <= 1024:
        nat0 = torch.from_numpy(np.ascontiguousarray(e.natives[0].astype(np.float32))).to(dev)
        out_g = torch.empty((N, 3), dtype=torch.float32, device=dev)
        g = timer(lambda: clusco.gdt_tm_vs_ref(X, nat0, out=out_g), 3, 1)
        status("the GDT / TM-score calls")
        g_ms = max_over_ranks([statistics.mean(g["ms"])], dev, ws_)[0]
        g_err, g_cpu = None, None
        if rank == 0:
            import oracle
            idx = np.random.default_rng(7).choice(N, min(N, 200), replace=False)
            t0 = time.perf_counter()
            want = oracle.gdt_tm_vs_ref(e.coords[idx], e.natives[0].astype(np.float32))
            dt = time.perf_counter() - t0
            g_err = float(np.abs(out_g.cpu().numpy()[idx].astype(np.float64) - want).max())
            g_cpu = {"value": len(idx) / dt, "unit": "models/s", "cores": oracle.max_threads(), "kind": "oracle",
                     "sample": f"{len(idx)} sampled models against the native, {dt:.1f} s"}
        line["gdt_tm_vs_ref"] = {"workload": wl, "value": whole_job_rate(N, g_ms, ws_), "unit": "models/s",
                                 "ms": g_ms, "scores": "GDT_TS, TM-score, MaxSub", "reference": "first native",
                                 "max_abs_diff_sampled": g_err, "cpu_baseline": g_cpu,
                                 "bound": "issue latency (per-atom distances in FP32; FP64 for each superposition's "
                                          "solve and for the distances near a cutoff)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
