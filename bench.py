#!/usr/bin/env python3
"""Benchmark: all-vs-all cRMSD pairs/s (forward, forward+backward) on one B300.

Workload (default): N = 5,000 models x L = 300 atoms, 5 seeded natives x 1,000 models,
sigma ~ U(0.5, 10) A, random rigid motions (the plain-method-at-scale ensemble). One step
is one pass of the whole hot path over that ensemble:
    pre-pass + all-pairs forward (12,497,500 pairs, condensed FP32 matrix)
    + one-versus-native scoring of all 5,000 models
    + the adjoint of sum_ab w_ab cRMSD_ab (w ~ U[0,1], fixed) to d/dcoords.
``value`` is pairs per second of that step (P / step time, device time by CUDA events,
inputs resident in HBM). L2 is flushed (a 512 MiB write) before every timed step, outside
the events. ``e2e`` repeats the step through the public API with host buffers: the
step's inputs go host->device from pinned memory and the matrix, the vs-native scores and
the gradient come back device->host inside the timed region.

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
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "all-vs-all cRMSD pairs/s (fwd+bwd step) at max err <= 1e-3 A"
UNIT = "pairs/s"


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--form", default=None, help="fp32_simt | tf32 | bf16x3 | bf16_exact2 (default: best built)")
    p.add_argument("--N", type=int, default=5000)
    p.add_argument("--L", type=int, default=300)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-drmsd", action="store_true",
                   help="skip the dRMSD, contact map overlap and GDT / TM-score measurements")
    p.add_argument("--cpu-models", type=int, default=5000, help="models in the oracle's timed sample")
    p.add_argument("--ref-models", type=int, default=800, help="models per step of the reference arm")
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
    from paper_1302_4000_b300 import ensembles as E
    e = E.config1(N=N, L=L)
    w = E.weights(N * (N - 1) // 2, E.SEED_BASE + 101)
    native = e.natives[0].astype(np.float32)
    return e, w, native


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


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


def traffic_for(key, N, L):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or None for another
    workload than the one captured (N models of L atoms) or once any library source has changed
    since the counters were taken (csrc_hash recorded beside them)."""
    try:
        h = csrc_hash()
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            parts = line.split()
            if (len(parts) == 6 and parts[0] == key and parts[1] == h and int(parts[2]) == N
                    and int(parts[3]) == L):
                return float(parts[4])
    except (OSError, ValueError):
        pass
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, 1400.0, "fallback"


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
    oracle.crmsd_grad(X, ws, 1e-6)
    dt = time.perf_counter() - t0
    P = n * (n - 1) // 2
    return {"value": P / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {P} pairs among the first {n} models (fwd + vs-native + gradient), {dt:.1f} s"}


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
            "config": {"workload": f"decoy ensemble N={args.N} L={args.L} (bounded sample: {n} models per step)",
                       "l2": "n/a (CPU)"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": times[0]["cores"], "kind": "oracle",
                             "sample": times[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    if args.form is None:
        form_name = "bf16_exact2"
        try:
            Xt = torch.zeros((4, 8, 3), device=dev)
            Xt[:, :, 0] = torch.arange(8, device=dev)
            clusco.crmsd_allpairs(Xt, clusco.FORM_BF16_EXACT2)
            torch.cuda.synchronize()
        except clusco.ClusCoError:
            form_name = "fp32_simt"
    else:
        form_name = args.form
    form = clusco.FORMS[form_name]

    e, w, native = workload(args.N, args.L)
    N, L = e.N, e.L
    P = N * (N - 1) // 2
    X = torch.from_numpy(e.coords).to(dev)
    W = torch.from_numpy(w).to(dev)
    ref = torch.from_numpy(native).to(dev)
    out = torch.empty(P, dtype=torch.float32, device=dev)
    vs = torch.empty(N, dtype=torch.float32, device=dev)
    grad = torch.empty_like(X)
    # the training step's path: with a tensor-core form and L <= 512 the forward stores each
    # pair's rotation and the adjoint contracts from it; otherwise the adjoint recomputes
    use_rot = form != clusco.FORM_FP32_SIMT and L <= 512
    rot = torch.empty((P, clusco.ROT_STRIDE), dtype=torch.float32, device=dev) if use_rot else None
    ws_all = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS_ROT if use_rot else clusco.OP_ALLPAIRS, N, L,
                                                form), dtype=torch.uint8, device=dev)
    ws_vs = torch.empty(clusco.workspace_bytes(clusco.OP_VS_REF, N, L, form), dtype=torch.uint8, device=dev)
    ws_bw = torch.empty(clusco.workspace_bytes(clusco.OP_BACKWARD_ROT if use_rot else clusco.OP_BACKWARD, N, L,
                                               form), dtype=torch.uint8, device=dev)

    def forward(Xd, o=None, st=None):
        o = out if o is None else o
        if use_rot:
            clusco.crmsd_allpairs_rot(Xd, form, out=o, rot=rot, workspace=ws_all, stream=st)
        else:
            clusco.crmsd_allpairs(Xd, form, out=o, workspace=ws_all, stream=st)

    def backward(Xd, Wd, o=None, gr=None, st=None):
        o = out if o is None else o
        gr = grad if gr is None else gr
        if use_rot:
            clusco.crmsd_allpairs_backward_rot(Xd, Wd, o, rot, 1e-6, grad_coords=gr, workspace=ws_bw, stream=st)
        else:
            clusco.crmsd_allpairs_backward(Xd, Wd, o, 1e-6, form, grad_coords=gr, workspace=ws_bw, stream=st)
    # the fused step (forward, then the adjoint from its rotations, in one call: the adjoint's
    # pre-pass runs beside the forward on the library's own stream)
    ws_st = (torch.empty(clusco.workspace_bytes(clusco.OP_STEP_ROT, N, L, form), dtype=torch.uint8, device=dev)
             if use_rot else None)

    def fused(Xd, Wd, o=None, gr=None, st=None):
        clusco.crmsd_allpairs_step_rot(Xd, Wd, form, 1e-6, out=out if o is None else o, rot=rot,
                                       grad_coords=grad if gr is None else gr, workspace=ws_st, stream=st)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # one-versus-native needs neither the forward nor the adjoint: it runs on a second stream,
    # forked at the start of the step and joined before its end, so that its small kernels fill
    # the SMs the forward's tail and the adjoint's pre-pass leave idle (the step's time is that
    # of both streams; "fwd" is the forward with that work beside it)
    side = torch.cuda.Stream()
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step_split(evs=None):
        # the two calls in turn, with events between them: the forward / adjoint breakdown
        if evs:
            evs[0].record(stream)
        fork.record(stream)
        side.wait_event(fork)
        clusco.crmsd_vs_ref(X, ref, out=vs, workspace=ws_vs, stream=side)
        join.record(side)
        forward(X)
        if evs:
            evs[1].record(stream)
            evs[2].record(stream)
        backward(X, W)
        stream.wait_event(join)
        if evs:
            evs[3].record(stream)

    def step():
        # the timed step: the fused call where rotations are stored, else the two calls
        if not use_rot:
            return step_split()
        fork.record(stream)
        side.wait_event(fork)
        clusco.crmsd_vs_ref(X, ref, out=vs, workspace=ws_vs, stream=side)
        join.record(side)
        fused(X, W)
        stream.wait_event(join)

    # our kernels per step: forward (pre-pass + pairs, + the refinement of flagged pairs in the
    # exact-digit form, + the deferred-rotation kernel when storing rotations); ref pre-pass + vs-ref; adjoint from stored rotations (pre-pass, FP16
    # split, max |w|, sweep, reduce, near-duplicate pass), or recomputing (pre-pass, transpose,
    # sweep, reduce, near-duplicate pass; 3 kernels on the CUDA-core adjoint)
    tc_bwd = L <= 320 and form != clusco.FORM_FP32_SIMT
    exact2 = form == clusco.FORM_BF16_EXACT2  # its forward adds the refinement of flagged pairs
    launches_per_step = (3 if use_rot else 2) + int(exact2) + 2 + (6 if use_rot else (5 if tc_bwd else 3))

    def timed(fn, k, w_, split=False, prof=False):
        for _ in range(w_):
            fn()
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k)]
        if ws_ > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if prof:  # the library brackets each tensor-core kernel launch with events on its stream
            clusco.profile_enable(True)
        for e4 in ev:
            flush.fill_(1)
            if split:
                fn(e4)
            else:
                e4[0].record(stream)
                fn()
                e4[3].record(stream)
        torch.cuda.synchronize()
        if prof:
            clusco.profile_enable(False)
        if ws_ > 1:
            dist.barrier()
        tot = [e4[0].elapsed_time(e4[3]) for e4 in ev]
        if not split:
            return tot, None, None
        return tot, [e4[0].elapsed_time(e4[1]) for e4 in ev], [e4[2].elapsed_time(e4[3]) for e4 in ev]

    clocks = Clocks(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    step_ms = timed(step, args.steps, args.warmup, prof=True)[0]
    clk = clocks.stop()
    # per-launch device time of the two tensor-core kernels inside the timed steps
    kern = {}
    for name, kid in (("pairs", clusco.KERNEL_PAIRS), ("adjoint", clusco.KERNEL_ADJOINT)):
        tot_ms, n = clusco.profile_read(kid)
        kern[name] = (tot_ms / n, n) if n else (None, 0)
    if clusco.sync_status() != 0:
        raise RuntimeError("device status set during the timed steps: " + lib.clusco_last_error().decode())
    _, fwd_list, bwd_list = timed(step_split, max(3, args.steps // 4), 2, split=True)
    ms = statistics.mean(step_ms)
    fms = statistics.mean(fwd_list)
    bms = statistics.mean(bwd_list)
    ms, fms, bms = max_over_ranks([ms, fms, bms], dev, ws_)

    # plain-form forward for the "vs plain FP32" ratio (same GPU, same inputs)
    plain_fwd = None
    if form != clusco.FORM_FP32_SIMT:
        ws_p = torch.empty(clusco.workspace_bytes(clusco.OP_ALLPAIRS, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                           device=dev)
        out_p = torch.empty_like(out)

        def pfwd():
            clusco.crmsd_allpairs(X, clusco.FORM_FP32_SIMT, out=out_p, workspace=ws_p)
        plain_fwd = statistics.mean(timed(pfwd, max(2, args.steps // 2), 1)[0])
        del ws_p, out_p

    # accuracy of this run's output on sampled pairs against the oracle (outside timing)
    max_err = None
    if rank == 0:
        import oracle
        rng = np.random.default_rng(3)
        ia = rng.integers(0, N, 4000)
        ib = rng.integers(0, N, 4000)
        keep = ia != ib
        ia, ib = np.minimum(ia[keep], ib[keep]), np.maximum(ia[keep], ib[keep])
        idx = ia * N - ia * (ia + 1) // 2 + (ib - ia - 1)
        got = out.cpu().numpy()[idx].astype(np.float64)
        want = oracle.crmsd_pairs(e.coords, ia, ib)
        max_err = float(np.abs(got - want).max())

    # e2e through the public API with host buffers. Each step copies its inputs (coords,
    # weights, native) host -> device from pinned memory and its results (matrix, vs-native
    # scores, gradient) back, all inside the timed region. Steps are pipelined the way a user
    # streaming ensembles would run them: three device buffer sets, the uploads of step k+1 and
    # the downloads of step k-1 on their own streams overlap the compute of step k (with two
    # sets, step k+1's uploads would wait for step k-1's downloads, which start only when its
    # compute ends). Throughput
    # = steps / (first upload start .. last download end). The working set (the stored
    # rotations alone are 48 B per pair) is far larger than L2, so no flush between steps.
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(e.coords).pin_memory()
        Wh = torch.from_numpy(w).pin_memory()
        Rh = torch.from_numpy(native).pin_memory()
        out_h = torch.empty(P, dtype=torch.float32).pin_memory()
        vs_h = torch.empty(N, dtype=torch.float32).pin_memory()
        g_h = torch.empty(X.shape, dtype=torch.float32).pin_memory()
        nbuf = 3  # step k+1's uploads need step k-2's downloads done, so copies never wait on compute
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
                    if k >= nbuf:  # this buffer set's previous results are on the host and its inputs consumed
                        s_in.wait_event(b["copied"])
                    b["X"].copy_(Xh, non_blocking=True)
                    b["W"].copy_(Wh, non_blocking=True)
                    b["R"].copy_(Rh, non_blocking=True)
                    b["in_ready"].record(s_in)
                s_cmp.wait_event(b["in_ready"])
                s_vs.wait_event(b["in_ready"])
                clusco.crmsd_vs_ref(b["X"], b["R"], out=b["vs"], workspace=ws_vs, stream=s_vs)
                b["vs_done"].record(s_vs)
                # the two calls in turn: with the host link the bound here, the fused call's side
                # stream measured 1.2 % slower per step (1.911 against 1.888 ms) in this pipeline
                forward(b["X"], o=b["out"], st=s_cmp)
                backward(b["X"], b["W"], o=b["out"], gr=b["g"], st=s_cmp)
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
        # The host link's own rates with the same pinned buffers (the weights up, the matrix
        # down): one direction at a time, then both at once, as the pipelined steps run them.
        # With both directions busy the step cannot take less than its larger byte count at
        # the concurrent rate.
        b0 = bufs[0]
        up = lambda: b0["W"].copy_(Wh, non_blocking=True)
        down = lambda: out_h.copy_(b0["out"], non_blocking=True)

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
        l_up = link_gbs([(s_in, up)])
        l_down = link_gbs([(s_out, down)])
        l_both = link_gbs([(s_in, up), (s_out, down)])
        e2e = {"value": whole_job_rate(P, e_ms, ws_), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e_ms,
               "pipelined": "three buffer sets; uploads of step k+1 and downloads of step k-1 overlap step k",
               "calls": "forward and backward in turn (the faster of the two public paths here)",
               "l2": "working set larger than L2, no flush",
               "link_GBs": {"h2d": l_up, "d2h": l_down, "each_way_when_both": l_both,
                            "floor_ms_per_step": max(h2d, d2h) / (l_both * 1e6)}}
        del bufs

    hbm, bf16, bf16_sus, pk_kind = peaks()
    # All-versus-all dRMSD (eq. 5) on the same ensemble: the tensor-core form (exact Gram of the
    # 16-bit rounded distances) against the plain FP32 form, L2 flushed before each call; the
    # contraction is 2 K flop per pair over K = L (L - 1) / 2 distances (one multiply-add per
    # atom pair), executed as four BF16 digit-product classes.
    drmsd = None
    if not args.no_drmsd and form == clusco.FORM_BF16_EXACT2 and 2 <= L <= 4096:
        K = L * (L - 1) // 2
        ws_d = torch.empty(clusco.workspace_bytes(clusco.OP_DRMSD, N, L, form), dtype=torch.uint8, device=dev)
        out_d = torch.empty(P, dtype=torch.float32, device=dev)

        def dfwd():
            clusco.drmsd_allpairs(X, clusco.FORM_BF16_EXACT2, out=out_d, workspace=ws_d)
        d_ms = statistics.mean(timed(dfwd, max(3, args.steps // 20), max(2, args.warmup), prof=True)[0])
        tot_ms, n = clusco.profile_read(clusco.KERNEL_DRMSD)
        dk_ms = tot_ms / n if n else None
        ws_dp = torch.empty(clusco.workspace_bytes(clusco.OP_DRMSD, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                            device=dev)
        out_dp = torch.empty_like(out_d)

        def dplain():
            clusco.drmsd_allpairs(X, clusco.FORM_FP32_SIMT, out=out_dp, workspace=ws_dp)
        dp_ms = statistics.mean(timed(dplain, 2, 1)[0])
        if clusco.sync_status() != 0:
            raise RuntimeError("device status set during the dRMSD calls: " + lib.clusco_last_error().decode())
        d_ms, dp_ms = max_over_ranks([d_ms, dp_ms], dev, ws_)
        d_err = None
        if rank == 0:
            import oracle
            rng = np.random.default_rng(4)
            ia = rng.integers(0, N, 4000)
            ib = rng.integers(0, N, 4000)
            keep = ia != ib
            ia, ib = np.minimum(ia[keep], ib[keep]), np.maximum(ia[keep], ib[keep])
            idx = ia * N - ia * (ia + 1) // 2 + (ib - ia - 1)
            d_err = float(np.abs(out_d.cpu().numpy()[idx].astype(np.float64)
                                 - oracle.drmsd_pairs(e.coords, ia, ib)).max())
        kms = dk_ms if dk_ms else d_ms
        ach = 2.0 * K * P / (kms * 1e-3) / 1e12
        Npad = (N + 127) // 128 * 128
        tiles = (Npad // 128) * (Npad // 64) - (Npad // 128) * (Npad // 128 - 1)
        executed = 4 * 2.0 * ((K + 63) // 64 * 64) * 128 * 64 * tiles  # digit classes, padded K, whole tiles
        drmsd = {"value": whole_job_rate(P, d_ms, ws_), "unit": UNIT, "ms": d_ms, "form": "bf16_exact2",
                 "vs_plain_fp32": dp_ms / d_ms, "plain_fp32_ms": dp_ms, "max_err_sampled_A": d_err,
                 "roofline": {"kernel": "drmsd_tc_kernel (Gram of the rounded distances, 2 K flop/pair)",
                              "launch_ms": kms, "timing": "kernel launch events" if dk_ms else "API call bracket",
                              "bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                              "frac": ach / bf16, "peak_kind": f"{pk_kind} bf16 burst",
                              "executed_tflops": executed / (kms * 1e-3) / 1e12,
                              "traffic": traffic_for("drmsd_tc", N, L)}}
        del ws_d, out_d, ws_dp, out_dp

    # All-versus-all contact map overlap (eq. 6, eq. 7) at an 8 A cutoff: the tensor-core form
    # (E4M3 0/1 maps, kind::f8f6f4) against the plain bit-count form. The contraction is 2 K flop
    # per pair (n(A and B) over K atom pairs); its peak is the FP8 rate, twice the measured BF16.
    cmo = None
    if not args.no_drmsd and form == clusco.FORM_BF16_EXACT2 and 2 <= L <= 4096:
        K = L * (L - 1) // 2
        ws_c = torch.empty(clusco.workspace_bytes(clusco.OP_CMO, N, L, clusco.FORM_FP8_EXACT), dtype=torch.uint8,
                           device=dev)
        out_c = torch.empty(P, dtype=torch.float32, device=dev)

        def cfwd():
            clusco.cmo_allpairs(X, 8.0, clusco.FORM_FP8_EXACT, out=out_c, workspace=ws_c)
        c_ms = statistics.mean(timed(cfwd, max(3, args.steps // 10), max(2, args.warmup), prof=True)[0])
        tot_ms, n = clusco.profile_read(clusco.KERNEL_CMO)
        ck_ms = tot_ms / n if n else None
        ws_cp = torch.empty(clusco.workspace_bytes(clusco.OP_CMO, N, L, clusco.FORM_FP32_SIMT), dtype=torch.uint8,
                            device=dev)
        out_cp = torch.empty_like(out_c)

        def cplain():
            clusco.cmo_allpairs(X, 8.0, clusco.FORM_FP32_SIMT, out=out_cp, workspace=ws_cp)
        cp_ms = statistics.mean(timed(cplain, 3, 1)[0])
        if clusco.sync_status() != 0:
            raise RuntimeError("device status set during the contact-map calls: " + lib.clusco_last_error().decode())
        c_ms, cp_ms = max_over_ranks([c_ms, cp_ms], dev, ws_)
        c_err = None
        if rank == 0:
            import oracle
            rng = np.random.default_rng(6)
            ia = rng.integers(0, N, 4000)
            ib = rng.integers(0, N, 4000)
            keep = ia != ib
            ia, ib = np.minimum(ia[keep], ib[keep]), np.maximum(ia[keep], ib[keep])
            idx = ia * N - ia * (ia + 1) // 2 + (ib - ia - 1)
            c_err = float(np.abs(out_c.cpu().numpy()[idx].astype(np.float64)
                                 - oracle.cmo_pairs(e.coords, ia, ib, 8.0)).max())
        kms = ck_ms if ck_ms else c_ms
        ach = 2.0 * K * P / (kms * 1e-3) / 1e12
        cmo = {"value": whole_job_rate(P, c_ms, ws_), "unit": UNIT, "ms": c_ms, "form": "fp8_exact", "cutoff_A": 8.0,
               "vs_plain_popcount": cp_ms / c_ms, "plain_popcount_ms": cp_ms, "max_err_sampled_pct": c_err,
               "roofline": {"kernel": "cmo_tc_kernel (Gram of the 0/1 contact maps, 2 K flop/pair)",
                            "launch_ms": kms, "timing": "kernel launch events" if ck_ms else "API call bracket",
                            "bound": "tensor", "achieved": ach, "peak": 2.0 * bf16, "unit": "TFLOP/s",
                            "frac": ach / (2.0 * bf16), "peak_kind": f"{pk_kind} bf16 burst x 2 (FP8 nominal ratio)",
                            "traffic": traffic_for("cmo_tc", N, L)}}
        del ws_c, out_c, ws_cp, out_cp

    # GDT_TS / TM-score / MaxSub of every model against its first native (eq. 3, eq. 4; the
    # paper's one-versus-reference use): the FP64 superposition search, timed as calls on the
    # resident ensemble, with the oracle on a bounded sample of models on the host cores.
    gdt = None
    if not args.no_drmsd and 3 <= L <= 1024:
        nat0 = torch.from_numpy(np.ascontiguousarray(native)).to(dev)
        out_g = torch.empty((N, 3), dtype=torch.float32, device=dev)

        def gfwd():
            clusco.gdt_tm_vs_ref(X, nat0, out=out_g)
        g_ms = statistics.mean(timed(gfwd, 3, 1)[0])
        if clusco.sync_status() != 0:
            raise RuntimeError("device status set during the GDT / TM-score calls: " + lib.clusco_last_error().decode())
        g_ms = max_over_ranks([g_ms], dev, ws_)[0]
        g_err, g_cpu = None, None
        if rank == 0:
            import oracle
            idx = np.random.default_rng(7).choice(N, min(N, 200), replace=False)
            t0 = time.perf_counter()
            want = oracle.gdt_tm_vs_ref(e.coords[idx], native)
            dt = time.perf_counter() - t0
            g_err = float(np.abs(out_g.cpu().numpy()[idx].astype(np.float64) - want).max())
            g_cpu = {"value": len(idx) / dt, "unit": "models/s", "cores": oracle.max_threads(), "kind": "oracle",
                     "sample": f"{len(idx)} sampled models against the native, {dt:.1f} s"}
        gdt = {"value": whole_job_rate(N, g_ms, ws_), "unit": "models/s", "ms": g_ms,
               "scores": "GDT_TS, TM-score, MaxSub", "reference": "first native",
               "max_abs_diff_sampled": g_err, "cpu_baseline": g_cpu,
               "bound": "issue latency (per-atom distances in FP32; FP64 for each superposition's solve and "
                        "for the distances near a cutoff)"}
        del out_g

    # Rooflines of the two tensor-core kernels. Algorithmic flop per pair: the forward
    # contraction is 18 L (the 3x3 covariance over L atoms); the adjoint is 54 L (that
    # covariance once, plus R x_b and R^T x_a over L atoms for the two gradients). One launch
    # of either kernel covers all P pairs. Duration: the kernel's own launch, bracketed by
    # events the library records on the launch stream during the timed steps (average over
    # the steps); the call bracket only where the kernel did not run (CUDA-core forms).
    def rf(flop, kms, call_ms, kernel, hash_key, hbm_bytes=None):
        msec = kms if kms else call_ms
        r = {"kernel": kernel, "launch_ms": msec, "timing": "kernel launch events" if kms else "API call bracket",
             "traffic": traffic_for(hash_key, N, L)}
        if hbm_bytes is None:
            ach = flop / (msec * 1e-3) / 1e12
            r.update({"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                      "peak_kind": f"{pk_kind} bf16 burst"})
        else:
            ach = hbm_bytes / (msec * 1e-3) / 1e9
            r.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                      "peak_kind": f"{pk_kind} HBM copy"})
        return r
    kp, ka = kern["pairs"][0], kern["adjoint"][0]
    if use_rot:
        # storing rotations, the forward writes 52 bytes per pair (the 48-byte rotation record and
        # the 4-byte cRMSD) against 18 L flop: at this L the HBM term of the roofline is the larger
        r_fwd = rf(18.0 * L * P, kp, fms, "pairs_tc_kernel<ROT> (forward storing rotations, 52 B/pair)",
                   "pairs_tc_rot", hbm_bytes=52.0 * P)
    else:
        r_fwd = rf(18.0 * L * P, kp, fms, "pairs_tc_kernel (forward, 18 L flop/pair)", "pairs_tc")
    if use_rot:
        # from stored rotations the adjoint's contraction is 36 L flop per pair (R x_b and R^T x_a)
        # against 44 bytes per pair of gathers (the nine floats of R_ab, c_ab, w_ab): the HBM
        # term is the larger
        r_bwd = rf(36.0 * L * P, ka, bms, "bwd_rot_kernel (adjoint from stored rotations, 44 B/pair)", "bwd_rot",
                   hbm_bytes=44.0 * P)
    else:
        r_bwd = rf(54.0 * L * P, ka, bms, "bwd_tc_kernel (adjoint, 54 L flop/pair)", "bwd_tc")
    dominant, other = (r_bwd, r_fwd) if r_bwd["launch_ms"] >= r_fwd["launch_ms"] else (r_fwd, r_bwd)
    line = {"metric": METRIC, "value": whole_job_rate(P, ms, ws_), "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32_simt": "f32+f64", "tf32": "tf32+f32",
                                           "bf16x3": "bf16+f32", "bf16_exact2": "bf16(exact int)+f32/f64"}[form_name],
            "data": "synthetic",
            "config": {"workload": f"decoy ensemble N={N} L={L}, 5 natives, sigma~U(0.5,10) A", "form": form_name,
                       "pairs": P,
                       "step": ("prepass + all-pairs fwd + vs-native + backward"
                                + (" (fwd and backward in one call, the backward's pre-pass beside the fwd; fwd and"
                                   " bwd_ms from the two calls in turn)" if use_rot else "")),
                       "adjoint": "from stored rotations" if use_rot else "recomputed covariances",
                       "l2": "flushed (512 MiB write) before each timed step", "parallelism": f"replicas x{ws_}"},
            "fwd": {"value": whole_job_rate(P, fms, ws_), "unit": UNIT, "ms": fms},
            "bwd_ms": bms,
            "vs_plain_fp32_fwd": (plain_fwd / fms) if plain_fwd else 1.0,
            "plain_fp32_fwd_ms": plain_fwd,
            "max_err_sampled_A": max_err,
            "roofline": dominant, "roofline_other": other,
            "clocks": clk, "gpu_launches": launches_per_step * args.steps}
    if e2e:
        line["e2e"] = e2e
    if drmsd:
        line["drmsd"] = drmsd
    if cmo:
        line["cmo"] = cmo
    if gdt:
        line["gdt_tm_vs_ref"] = gdt
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(e, w, native, args.cpu_models)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
