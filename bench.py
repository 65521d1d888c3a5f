#!/usr/bin/env python3
"""Benchmark of the state-vector gate engine on GB300.

One step = one pass of the hot path over the 30-qubit complex128 workload:
  HALL on |0..0> (the step's input state; qc_hall, n Hadamards in fused
  tile passes), 100 Grover iterations with 8 seeded marked items (oracle +
  diffusion, one fused pass each), the QFT, the Born-rule probabilities and
  1000 seeded samples, then the per-gate sweep H(t), CNOT((t+1) mod n, t),
  CPHASE((t+1) mod n, t, k=1) for t = 0..n-1.  In the device-timed loop
  each step first writes its input |0..0> (qc_state_reset, inside the timed
  region); the end-to-end loop uploads it from host memory instead.
Metric: amplitude-updates/s = 2^n x (operators applied per step) / step
time, where HALL, each Grover operator G, the QFT and each swept gate count
as one operator acting on all 2^n amplitudes (192 operators per step at
n = 30).  The state (16 GiB) is larger than L2, so no flush is needed.

Extra keys report the per-kernel bandwidth table, the 32-qubit complex64
workload, the 10-qubit Grover run, the 24-qubit random circuit, the
batched noisy trajectories and the adjoint gradient (each measured outside
the timed region).

Under torchrun with N > 1 every rank runs an independent replica (the path
does not shard in this build); value = the work of all ranks / the slowest
rank's time.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-updates/s & HBM GB/s per gate (30q); adjoint grad time/forward"
UNIT = "amp-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30, help="qubits of the main workload")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"], help="state type of the main workload")
    ap.add_argument("--iters", type=int, default=100, help="Grover iterations per step")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", default="", help="run just one extra (profiling helper)")
    return ap.parse_args()


# ----------------------------------------------------------- distributed ----

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(times_ms, work_units, backend_group=None):
    """Whole-job value from per-rank elapsed times: work of all ranks / the
    slowest rank's time.  Uses torch.distributed when initialised."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([times_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        w = torch.tensor([work_units], dtype=torch.float64, device=dev)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        return float(t.item()), float(w.item())
    return float(times_ms), float(work_units)


# ---------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- our arm ----

def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_0902_0699_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(profile_name, src_hash):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", profile_name)
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha", "").split(" ")[0] != src_hash:
        return None
    try:
        return float(vals["traffic_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class Events:
    def __init__(self, torch):
        self.torch = torch
        self.ev = []

    def mark(self, name):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record()
        self.ev.append((name, e))

    def spans(self):
        out = {}
        for (a, ea), (b, eb) in zip(self.ev, self.ev[1:]):
            out.setdefault(b, 0.0)
            out[b] += ea.elapsed_time(eb)
        return out


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_0902_0699_gb300 as qc
    import workloads as W

    torch.cuda.set_device(local)
    n, iters = args.n, args.iters
    N = 1 << n
    amp = 16 if args.dtype == "c128" else 8
    S = N * amp
    marked = W.marked_indices(W.rng(2026), n, 8)
    st = qc.State(n, qc.QC_C128 if args.dtype == "c128" else qc.QC_C64)
    H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    ops_per_step = 1 + iters + 1 + 3 * n

    def step(ev: Events | None, sweep_ev=None, state=None):
        # state: an uploaded |0..0> (end-to-end loop); else write it here
        st_ = state if state is not None else st
        if ev: ev.mark("start")
        if state is None:
            st_.reset(0)
        if ev: ev.mark("input_reset")
        st_.hall()
        if ev: ev.mark("hall")
        for _ in range(iters):
            st_.grover_step(marked)
        if ev: ev.mark("grover")
        st_.qft()
        if ev: ev.mark("qft")
        _, shots = st_.probs_sample(12345, 1000)  # probabilities and samples from one read
        if ev: ev.mark("probs_sample")
        for t in range(n):
            if sweep_ev is not None: sweep_ev[("h", t)][0].record()
            st_.apply_1q(t, H)
            if sweep_ev is not None:
                sweep_ev[("h", t)][1].record()
                sweep_ev[("cnot", t)][0].record()
            st_.cnot((t + 1) % n, t)
            if sweep_ev is not None:
                sweep_ev[("cnot", t)][1].record()
                sweep_ev[("cphase", t)][0].record()
            st_.cphase((t + 1) % n, t, 1)
            if sweep_ev is not None: sweep_ev[("cphase", t)][1].record()
        if ev: ev.mark("sweep")
        return shots

    import torch.distributed as dist
    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    if dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    launches0 = qc.kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    evs = []
    sweep_all = []
    t0.record()
    for _ in range(args.steps):
        ev = Events(torch)
        sw = {(g, t): (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for g in ("h", "cnot", "cphase") for t in range(n)}
        step(ev, sw)
        evs.append(ev)
        sweep_all.append(sw)
    t1.record()
    torch.cuda.synchronize()
    if dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    launches = qc.kernel_launches() - launches0
    clocks = clk.stop()
    elapsed = t0.elapsed_time(t1)
    work = float(ops_per_step) * N * args.steps
    tmax, wsum = aggregate(elapsed, work)
    value = wsum / (tmax / 1e3)

    # component times (mean per step, ms)
    comp = {}
    for ev in evs:
        for k, v in ev.spans().items():
            comp[k] = comp.get(k, 0.0) + v / args.steps
    sweep = {}
    for g in ("h", "cnot", "cphase"):
        per_t = [statistics.mean(sw[(g, t)][0].elapsed_time(sw[(g, t)][1]) for sw in sweep_all) for t in range(n)]
        sweep[g] = per_t
    bytes_gate = {"h": 2 * S, "cnot": S, "cphase": S // 2}
    peak = read_peaks()
    hbm = peak["hbm_gbs"]
    gb = lambda b, ms: b / (ms * 1e-3) / 1e9
    grover_ms = comp["grover"] / iters
    kernels = {
        "grover_step (prep+pass+fix)": {"ms": grover_ms, "alg_bytes": 2 * S, "GB/s": gb(2 * S, grover_ms),
                                        "launches_per_step": iters * 3},
        "input_reset (|0..0>)": {"ms": comp["input_reset"], "alg_bytes": S, "GB/s": gb(S, comp["input_reset"])},
        "hall": {"ms": comp["hall"], "alg_bytes": hall_bytes(n, amp), "GB/s": gb(hall_bytes(n, amp), comp["hall"])},
        "qft": {"ms": comp["qft"], "alg_bytes": qft_bytes(n, amp), "GB/s": gb(qft_bytes(n, amp), comp["qft"])},
    }
    sweep_table = {}
    for g in ("h", "cnot", "cphase"):
        ms = sweep[g]
        sweep_table[g] = {"ms_mean": statistics.mean(ms), "GB/s_per_t": [round(gb(bytes_gate[g], m), 1) for m in ms],
                          "amp_updates_per_s_mean": N / (statistics.mean(ms) * 1e-3),
                          "frac_of_measured_min": round(min(gb(bytes_gate[g], m) for m in ms) / hbm, 3),
                          "frac_of_measured_max": round(max(gb(bytes_gate[g], m) for m in ms) / hbm, 3)}
    # dominant kernel: the fused Grover pass (100 launches per step)
    src_hash = kernel_source_hash(["grover.cu", "common.cuh", "ff.cuh"])
    traffic = read_traffic("grover_pass_n30_c128.txt", src_hash) if args.dtype == "c128" and n == 30 else None
    achieved = gb(2 * S, grover_ms)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "kernel": "k_grover_pass_%s (one fused oracle+diffusion read/write pass)" % args.dtype,
                "alg_bytes_per_launch": 2 * S, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    # accuracy of this workload, outside the timed region: HALL, the Grover
    # iterations and the QFT once more, against the closed form
    st.reset(0)
    st.hall()
    for _ in range(iters):
        st.grover_step(marked)
    st.qft()
    accuracy = error_vs_closed_form(st, n, marked, iters)
    accuracy["tolerance_abs"] = 1e-12 if args.dtype == "c128" else 1e-5
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 (f64 storage; f64 and double-float arithmetic)" if args.dtype == "c128" else "c64 (f32; f64 reductions)",
        "data": "synthetic",
        "config": {"workload": "grover%d_qft_sweep_%s" % (n, args.dtype), "qubits": n, "state_bytes": S,
                   "grover_iterations": iters, "marked": 8, "sweep": "H, CNOT(t+1 mod n, t), CPHASE k=1 for t=0..n-1",
                   "operators_per_step": ops_per_step,
                   "l2": "inputs larger than L2 (%.1f GiB state)" % (S / 2 ** 30) if S > 2 ** 27 else "state fits in L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline, "clocks": clocks, "gpu_launches": int(launches), "accuracy": accuracy,
        "kernels": kernels, "sweep": sweep_table, "component_ms_per_step": comp,
    }
    return out, st, step, ops_per_step, N


def hall_bytes(n, amp):
    """Algorithmic bytes of HALL as built: one read+write pass per tile
    group (csrc/tile.cu plan_groups)."""
    BOT, K = (12, 9) if amp == 16 else (13, 10)
    g0 = min(n, BOT)
    rest = n - g0
    passes = 1 + (-(-rest // K) if rest > 0 else 0)
    return passes * 2 * (1 << n) * amp


def grover_qft_closed_form(n, marked, k, idx):
    """Amplitudes of QFT(G^k HALL|0..0>) at indices idx, from the closed form
    (sec. 5.1 and the DFT identity of App. A): with theta = asin(sqrt(M/N)),
    a = sin((2k+1) theta)/sqrt(M) on the marked items and
    b = cos((2k+1) theta)/sqrt(N-M) elsewhere,
    QFT[j] = b sqrt(N) [j = 0] + (a - b)/sqrt(N) sum_m e^{2 pi i m j / N}."""
    import numpy as np
    N = 1 << n
    M = len(marked)
    th = math.asin(math.sqrt(M / N))
    a = math.sin((2 * k + 1) * th) / math.sqrt(M)
    b = math.cos((2 * k + 1) * th) / math.sqrt(N - M)
    out = np.zeros(len(idx), dtype=np.complex128)
    for i, j in enumerate(idx):
        acc = 0j
        for m in marked:
            ang = 2.0 * math.pi * ((int(m) * int(j)) % N) / N
            acc += complex(math.cos(ang), math.sin(ang))
        out[i] = (a - b) / math.sqrt(N) * acc + (b * math.sqrt(N) if int(j) == 0 else 0.0)
    return out


def error_vs_closed_form(st, n, marked, k, seed=7, samples=4096):
    """max |d amp| and max |d amp| / |amp| of st (after HALL, k Grover
    iterations and the QFT) against the closed form, on the zero index, the
    marked items and seeded random indices."""
    import numpy as np
    import torch
    g = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0], np.asarray(marked, dtype=np.int64),
                                    g.integers(0, 1 << n, samples, dtype=np.int64)]))
    got = st.tensor[torch.as_tensor(idx, device=st.tensor.device)].cpu().numpy().astype(np.complex128)
    ref = grover_qft_closed_form(n, marked, k, idx)
    d = np.abs(got - ref)
    return {"max_abs": float(d.max()), "max_rel": float((d / np.abs(ref)).max()),
            "median_abs_amp": float(np.median(np.abs(ref))), "indices": int(len(idx)),
            "against": "closed form of QFT(G^%d HALL|0..0>) (sec. 5.1, App. A)" % k}


def qft_bytes(n, amp):
    """Algorithmic bytes of the QFT as built: one read+write pass per tile
    group plus the bit-reversal pass."""
    # lowest group up to BOT qubits, the others up to K (the QFT group plans of csrc/tile.cu)
    BOT, K = (12, 9) if amp == 16 else (13, 9)
    g0 = min(n, BOT)
    rest = n - g0
    passes = 1 + (-(-rest // K) if rest > 0 else 0)
    return (passes + 1) * 2 * (1 << n) * amp


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d.get("hbm_gbs", 6800.0)), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


def gpu_numa_node(dev):
    """NUMA node of the host memory next to GPU `dev`, from the GPU's PCI
    device in sysfs (None if unknown)."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    addrs = []
    if hasattr(p, "pci_bus_id"):
        addrs.append("%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, getattr(p, "pci_device_id", 0)))
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        if out:  # e.g. 00000009:01:00.0
            dom, rest = out.split(":", 1)
            addrs.append(("%04x" % int(dom, 16)) + ":" + rest.lower())
    except Exception:
        pass
    for a in addrs:
        try:
            node = int(open("/sys/bus/pci/devices/%s/numa_node" % a).read().strip())
            if node >= 0:
                return node, a
        except Exception:
            continue
    return None, (addrs[0] if addrs else None)


class HostBuffer:
    """Page-locked host memory for the end-to-end copies: an anonymous
    mapping advised to transparent huge pages (MADV_HUGEPAGE), first touched
    from a thread bound to the CPUs of the GPU's NUMA node and registered
    with cudaHostRegister, so that the pages sit next to the GPU and are
    mapped with a few large translations.  Falls back to torch's pinned
    allocator (cudaHostAlloc) where the registration fails.  (On the GB300
    boxes cudaHostAlloc memory copied at 210 GB/s host->device on a fresh
    box but at 16-85 GB/s once the box had run the GPU tests; the huge-page
    buffer kept 210 GB/s on such a box.)"""

    MADV_HUGEPAGE = 14

    def __init__(self, nbytes, node):
        import ctypes
        import mmap
        import torch
        self.nbytes, self.node = nbytes, node
        self.t = None
        self.buf = None
        self.addr = None
        cpus = None
        if node is not None:
            try:
                cpus = parse_cpulist(open("/sys/devices/system/node/node%d/cpulist" % node).read())
            except Exception:
                cpus = None
        old = os.sched_getaffinity(0)
        bound = False
        if cpus and cpus & old:
            os.sched_setaffinity(0, cpus & old)
            bound = True
        try:
            try:
                libc = ctypes.CDLL(None, use_errno=True)
                libc.madvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
                libc.memset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
                buf = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
                addr = ctypes.addressof(ctypes.c_char.from_buffer(buf))
                thp = libc.madvise(ctypes.c_void_p(addr), ctypes.c_size_t(nbytes), self.MADV_HUGEPAGE) == 0
                libc.memset(ctypes.c_void_p(addr), 0, ctypes.c_size_t(nbytes))  # first touch, bound thread
                if int(torch.cuda.cudart().cudaHostRegister(addr, nbytes, 0)) != 0:
                    raise RuntimeError("cudaHostRegister failed")
                self.buf, self.addr = buf, addr
                self.t = torch.frombuffer(buf, dtype=torch.uint8, count=nbytes)
                self.method = "anonymous mapping%s, first touch from %s, cudaHostRegister" % (
                    " with MADV_HUGEPAGE" if thp else "",
                    ("a thread bound to node %d's CPUs" % node) if bound else "an unbound thread")
            except Exception as e:
                self.t = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
                self.t.zero_()
                self.method = "cudaHostAlloc (registration of a huge-page mapping failed: %s)" % e
        finally:
            if bound:
                os.sched_setaffinity(0, old)

    def tensor(self, dtype, numel):
        return self.t.view(dtype)[:numel]

    def close(self):
        import torch
        self.t = None
        if self.addr is not None:
            torch.cuda.cudart().cudaHostUnregister(self.addr)
            self.addr = None
        if self.buf is not None:
            try:
                self.buf.close()
            except BufferError:
                pass  # a view is still alive: the mapping goes with the process
            self.buf = None


def parse_cpulist(txt):
    cpus = set()
    for part in txt.strip().split(","):
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def run_e2e(args, st, step_fn, ops_per_step, N):
    """Same workload through the public API, from a host input to a host
    result: every step copies its input state (|0..0>, held in pinned host
    memory) host->device, runs the whole step on it and reads its result,
    the 1000 measurement samples, back to pinned host memory.  Two device
    states are used in turn, so a step's upload overlaps the other state's
    step; the uploads go through one copy stream.  (On the GB300 machines' host
    link a single copy runs at about 210 GB/s host->device from a huge-page
    buffer, while two copies at once ran at 9-17 GB/s; the state itself is
    not read back: the step's result is its samples.)  The timed region
    holds every step's copies."""
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    n = args.n
    cdt = st.tensor.dtype
    amp = st.tensor.element_size()
    node, pci = gpu_numa_node(torch.cuda.current_device())
    hb = HostBuffer(N * amp, node)
    host = hb.tensor(cdt, N)
    host[0] = 1.0  # the input |0..0>
    host_shots = [torch.empty(1000, dtype=torch.int64, pin_memory=True) for _ in range(args.steps + 2)]
    comp = torch.cuda.current_stream()
    st2 = qc.State(n, st.dt)
    states = [st, st2]
    s_copy = torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    copies = []  # (start, end) events of the uploads, on the copy stream

    def upload(b):
        with torch.cuda.stream(s_copy):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s_copy)
            states[b].tensor.copy_(host, non_blocking=True)
            z.record(s_copy)
            copies.append((a, z))
            ev_in[b].record(s_copy)

    def pipeline(k):
        # copy stream: upload 0, upload 1, then after step i the upload for
        # step i + 2 into the same device state; the compute stream runs
        # the steps, each followed by the read-back of its samples
        upload(0)
        if k > 1:
            upload(1)
        for i in range(k):
            b = i % 2
            comp.wait_event(ev_in[b])
            qc.qc_state_invalidate(states[b].h)
            shots = step_fn(None, None, states[b])
            host_shots[i].copy_(shots, non_blocking=True)  # the step's result, device -> host
            ev_done[b].record(comp)
            if i + 2 < k:
                with torch.cuda.stream(s_copy):
                    s_copy.wait_event(ev_done[b])
                upload(b)
    pipeline(2)  # warm-up
    torch.cuda.synchronize()
    copies.clear()
    t0 = time.perf_counter()
    pipeline(args.steps)
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) * 1e3
    rates = [N * amp / (a.elapsed_time(z) * 1e-3) / 1e9 for a, z in copies]
    tmax, wsum = aggregate(el, float(ops_per_step) * N * args.steps)
    st2.close()
    pinned = {"gpu_pci": pci, "gpu_numa_node": node, "host_in": hb.method, "host_in_is_pinned": bool(host.is_pinned()),
              "host_out": "torch pinned (8 KB of samples per step)"}
    ok = all(int(t.min()) >= 0 and int(t.max()) < N for t in host_shots[:args.steps])
    del host
    hb.close()
    return {"value": wsum / (tmax / 1e3), "unit": UNIT, "h2d_bytes_per_step": N * amp,
            "d2h_bytes_per_step": 8 * 1000, "ms_per_step": tmax / args.steps,
            "h2d_GBps_seen": statistics.mean(rates) if rates else None,
            "h2d_GBps_each": [round(r, 1) for r in rates], "samples_in_range": ok,
            "host_buffers": pinned,
            "note": "per step: the input state |0..0> from pinned host memory to the device, the whole step on it, "
                    "its 1000 samples back to pinned host memory; two device states in turn, so each upload "
                    "overlaps the other state's step"}


# ---------------------------------------------------------------- extras ----

def extra_c64(n=32, iters=100):
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    N = 1 << n
    S = N * 8
    marked = W.marked_indices(W.rng(2027), n, 8)
    st = qc.State(n, qc.QC_C64)
    H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    res = {}

    def run(timed):
        ev = Events(torch)
        ev.mark("start")
        st.reset(0)
        ev.mark("input_reset")
        st.hall()
        ev.mark("hall")
        for _ in range(iters):
            st.grover_step(marked)
        ev.mark("grover")
        st.qft()
        ev.mark("qft")
        if timed:
            res["accuracy"] = error_vs_closed_form(st, n, marked, iters)
            res["accuracy"]["tolerance_abs"] = 1e-5
            ev.mark("accuracy")
        hs = []
        for t in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(); st.apply_1q(t, H); b.record()
            c_, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c_.record(); st.cnot((t + 1) % n, t); d.record()
            e_, f = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_.record(); st.cphase((t + 1) % n, t, 1); f.record()
            hs.append(((a, b), (c_, d), (e_, f)))
        ev.mark("sweep")
        torch.cuda.synchronize()
        return ev.spans(), hs
    run(False)
    spans, hs = run(True)
    gb = lambda b, ms: b / (ms * 1e-3) / 1e9
    ms = [[x[0].elapsed_time(x[1]) for x in h] for h in hs]
    spans.pop("accuracy", None)
    total = sum(spans.values())
    res.update({"qubits": n, "state_bytes": S, "ms_total": total,
           "amp_updates_per_s": (1 + iters + 1 + 3 * n) * N / (total * 1e-3),
           "grover_step_ms": spans["grover"] / iters, "grover_GB/s": gb(2 * S, spans["grover"] / iters),
           "qft_ms": spans["qft"], "qft_GB/s": gb(qft_bytes(n, 8), spans["qft"]),
           "hall_ms": spans["hall"], "hall_GB/s": gb(hall_bytes(n, 8), spans["hall"]),
           "h_GB/s_mean": statistics.mean(gb(2 * S, m[0]) for m in ms),
           "cnot_GB/s_mean": statistics.mean(gb(S, m[1]) for m in ms),
           "cphase_GB/s_mean": statistics.mean(gb(S / 2, m[2]) for m in ms)})
    st.close()
    del st
    torch.cuda.empty_cache()
    return res


def extra_rho64(n=13, B=64, reps=3):
    """The ensemble density matrix of B random complex64 states on the
    tensor cores (profiling helper): rho is 4^n x 8 bytes (512 MiB at
    n = 13, larger than L2)."""
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    g = torch.Generator(device="cuda")
    g.manual_seed(13)
    t = torch.randn(B << n, 2, dtype=torch.float32, device="cuda", generator=g)
    t = torch.view_as_complex(t).reshape(B, 1 << n)
    t /= t.abs().pow(2).sum(dim=1, keepdim=True).sqrt()
    P = np.full(B, 1.0 / B)
    N = 1 << n
    rho = torch.empty(N * N, dtype=torch.complex64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    qc.qc_density_matrix(t.data_ptr(), n, qc.QC_C64, B, P, rho.data_ptr(), s)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        qc.qc_density_matrix(t.data_ptr(), n, qc.QC_C64, B, P, rho.data_ptr(), s)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    tr = float(rho.view(N, N).diagonal().real.sum().item())
    return {"qubits": n, "universes": B, "ms": ms, "GB/s_written": N * N * 8 / (ms * 1e6),
            "trace_minus_1": tr - 1.0}


def extra_u2_sweep(n=30, dtype="c128", reps=1):
    """General one-qubit operators on every target t = 0..n-1 of an n-qubit
    state: a Haar-random U(2) (the general complex kind) and RY (the real
    kind).  One read+write pass each (2S algorithmic bytes)."""
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    dt = qc.QC_C128 if dtype == "c128" else qc.QC_C64
    S = (1 << n) * (16 if dt == qc.QC_C128 else 8)
    st = qc.State(n, dt)
    st.uniform()
    U = W.haar_u2(W.rng(2), n)
    c, s_ = math.cos(0.3), math.sin(0.3)
    RY = np.array([[c, -s_], [s_, c]], dtype=np.complex128)
    hbm = read_peaks()["hbm_gbs"]
    res = {}
    for name, mats in (("haar_u2", U), ("ry", [RY] * n)):
        st.apply_1q(0, mats[0])  # warm-up
        torch.cuda.synchronize()
        evs = []
        for t in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                st.apply_1q(t, mats[t])
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) / reps for a, b in evs]
        gbs = [2 * S / (m * 1e-3) / 1e9 for m in ms]
        res[name] = {"ms_mean": statistics.mean(ms), "GB/s_per_t": [round(x, 1) for x in gbs],
                     "frac_of_measured_min": round(min(gbs) / hbm, 3), "frac_of_measured_max": round(max(gbs) / hbm, 3),
                     "frac_of_measured_mean": round(statistics.mean(gbs) / hbm, 3)}
    res["state"] = {"qubits": n, "dtype": dtype, "state_bytes": S}
    st.close()
    del st
    torch.cuda.empty_cache()
    return res


def extra_c1():
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    n = 10
    marked = W.marked_indices(W.rng(0), n, 1)
    st = qc.State(n, qc.QC_C128)
    it = W.grover_iterations(n)
    for _ in range(3):
        st.grover_run(marked, it)
        st.sample(1, 1000)
    torch.cuda.synchronize()
    reps = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for r in range(reps):
        st.grover_run(marked, it)
        p = st.probs()
        st.sample(r, 1000)
    b.record()
    torch.cuda.synchronize()
    ps = float(p[int(marked[0])].item())
    return {"qubits": n, "iterations": it, "us_per_run": a.elapsed_time(b) / reps * 1e3,
            "p_success": ps, "p_success_closed_form": math.sin((2 * it + 1) * math.asin(2 ** -5)) ** 2,
            "note": "grover_run (one kernel, state in shared memory) + probs + 1000 samples (sampling syncs the stream once, to read the weight total)"}


def extra_red(reps=3):
    """One call of each reduction on a 1 GiB random state per type (26 qubits
    complex128, 27 qubits complex64): Born probabilities, 1000 samples, the
    norm and three Pauli expectations (diagonal, X-type, Y-type pairing);
    then probabilities and samples from one read (probs_sample).
    One warm-up pass calls each once, in that order, before the timed
    repeats (so a profiler's first seven launches per type are one of each
    kernel).  Times are CUDA-event averages; GB/s counts one read of the
    state (plus the probabilities written, for probs)."""
    import torch
    import paper_0902_0699_gb300 as qc
    out = {}
    for n, dt, name in [(26, qc.QC_C128, "c128"), (27, qc.QC_C64, "c64")]:
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        rdt = torch.float64 if dt == qc.QC_C128 else torch.float32
        t = torch.randn(2 << n, dtype=rdt, device="cuda", generator=g)
        t /= t.norm()
        st = qc.State(n, dt, tensor=torch.view_as_complex(t.view(-1, 2)).contiguous())
        del t
        sb = (1 << n) * (16 if dt == qc.QC_C128 else 8)
        calls = {"probs": (lambda: st.probs(), sb + 8 * (1 << n)),
                 "sample_1000": (lambda: st.sample(12345, 1000), sb),
                 "norm": (lambda: st.norm(), sb),
                 "expect_z": (lambda: st.expect_pauli(0, 5), sb),
                 "expect_x": (lambda: st.expect_pauli(1 << (n - 1), 0), sb),
                 "expect_y": (lambda: st.expect_pauli(1 << (n - 1), 1 << (n - 1)), sb),
                 "probs_sample_1000": (lambda: st.probs_sample(12345, 1000), sb + 8 * (1 << n))}
        for fn, _ in calls.values():  # one warm-up pass over all calls first
            fn()
        torch.cuda.synchronize()
        res = {}
        for key, (fn, nbytes) in calls.items():
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            res[key] = {"ms": ms, "GBps": nbytes / ms / 1e6}
        out["%s_n%d" % (name, n)] = res
        st.close()
        del st
        torch.cuda.empty_cache()
    out["note"] = ("norm and expect return a host scalar and sample reads the weight total, so those "
                   "calls include one stream sync each; the state (1 GiB) is larger than L2")
    return out


def extra_c2():
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    n, layers = 24, 200
    circ = W.random_circuit(n, layers, seed=24)
    res = {}
    for dt, name in ((qc.QC_C128, "c128"), (qc.QC_C64, "c64")):
        st = qc.State(n, dt).reset(0)

        def run():
            st.reset(0)
            for l in range(layers):
                st.apply_1q_layer(circ.U[l])
                for (c, t) in circ.cnot_pairs(l):
                    st.cnot(c, t)
            st.qft()
        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        ncnot = sum(len(circ.cnot_pairs(l)) for l in range(layers))
        gates = layers * n + ncnot + n * (n + 1) // 2 + n // 2
        amp = 16 if dt == qc.QC_C128 else 8
        S = (1 << n) * amp
        # algorithmic bytes gate by gate: a one-qubit gate reads and writes
        # every amplitude (2S), a CNOT the half it moves (S); the QFT as built
        alg = layers * n * 2 * S + ncnot * S + qft_bytes(n, amp)
        ref = st.tensor.clone()  # the gate-by-gate result, for the fused cross-check
        res[name] = {"ms": ms, "gates": gates, "gate_level_amp_updates_per_s": gates * (1 << n) / (ms * 1e-3),
                     "alg_GB/s": alg / (ms * 1e-3) / 1e9, "norm_error": abs(st.norm() - 1.0)}
        # the same circuit grouped into dense blocks (gate fusion); complex64
        # blocks of 5 qubits run on the tensor cores
        ops = []
        for l in range(layers):
            for q in range(n):
                ops.append((1, q, 0, 0, circ.U[l, q]))
            for (c, t) in circ.cnot_pairs(l):
                ops.append((2, c, t, 0, None))
        kmax, pad = (5, True) if dt == qc.QC_C64 else (3, False)
        t0 = time.perf_counter()
        plan = qc.FusedPlan(n, ops, kmax=kmax, pad=pad)
        t_plan = (time.perf_counter() - t0) * 1e3

        def run_fused():
            st.reset(0)
            plan.run(st.h)
            st.qft()
        run_fused()
        torch.cuda.synchronize()
        a.record()
        run_fused()
        b.record()
        torch.cuda.synchronize()
        msf = a.elapsed_time(b)
        nb, _ = plan.info()
        plan.close()
        res[name + "_fused"] = {"ms": msf, "blocks": nb, "block_qubits": kmax, "plan_ms_host_once": t_plan,
                               "gates": gates, "gate_level_amp_updates_per_s": gates * (1 << n) / (msf * 1e-3),
                               "speedup_vs_gate_by_gate": ms / msf, "norm_error": abs(st.norm() - 1.0),
                               "max_abs_diff_vs_gate_by_gate": float((st.tensor - ref).abs().max().item())}
        if dt == qc.QC_C64:
            # the tensor-core blocks shrink the state uniformly (about 7e-7
            # each, from their FP32 accumulation): one renormalisation after
            # the circuit removes it
            st.renormalize()
            res[name + "_fused"]["after_renormalize"] = {
                "norm_error": abs(st.norm() - 1.0),
                "max_abs_diff_vs_gate_by_gate": float((st.tensor - ref).abs().max().item())}
        del ref
        st.close()
    return res


def extra_c4(n_inst=4096, n_lo=12, n_hi=20, seed=4096, autotune=1):
    """Noisy Grover trajectories: n_inst instances with n ~ U{n_lo..n_hi}."""
    import ctypes
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    tb = W.trajectory_batch(n_inst, n_lo, n_hi, seed=seed)
    n_inst = len(tb.nq)
    nq = np.ascontiguousarray(tb.nq, dtype=np.int32)
    mk = np.ascontiguousarray(tb.marked, dtype=np.uint64)
    it = np.ascontiguousarray(tb.iters, dtype=np.int32)
    d = qc.TrajDesc(n_inst, nq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    mk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                    it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tb.seed, tb.thr_gate, tb.thr_readout,
                    tb.p_readout)
    plan = ctypes.c_void_p()
    s = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    rc = qc.lib().qc_traj_plan_create(ctypes.byref(d), ctypes.c_void_p(s), autotune, ctypes.byref(plan))
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    if rc:
        return {"error": qc.last_error()}
    ps = torch.empty(n_inst, dtype=torch.float64, device="cuda")
    pr = torch.empty_like(ps)
    oc = torch.empty(n_inst, dtype=torch.int64, device="cuda")
    ne = torch.empty(n_inst, dtype=torch.int32, device="cuda")
    out = qc.TrajOut(ps.data_ptr(), pr.data_ptr(), oc.data_ptr(), ne.data_ptr())
    qc.lib().qc_traj_plan_run(plan, ctypes.byref(out))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    rc = qc.lib().qc_traj_plan_run(plan, ctypes.byref(out))
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    info = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
    qc.lib().qc_traj_plan_info(plan, *[ctypes.byref(x) for x in info])
    qc.lib().qc_traj_plan_free(plan)
    psn = ps.cpu().numpy()
    amp_its = float(np.sum((2.0 ** tb.nq) * (tb.iters + 1)))
    hist, edges = np.histogram(psn, bins=10, range=(0, 1))
    return {"instances": n_inst, "ms": ms, "instances_per_s": n_inst / (ms * 1e-3),
            # error-free iterations need no pass (one affine map per run of them),
            # so this is the rate of the iteration-by-iteration equivalent
            "equivalent_amp_iterations_per_s": amp_its / (ms * 1e-3), "plan_s_with_autotune": t_plan,
            "shape": {"ctas_per_instance": info[0].value, "threads": info[1].value, "grid": info[2].value},
            "p_success_mean": float(psn.mean()), "p_readout_mean": float(pr.cpu().numpy().mean()),
            "errors_mean": float(ne.cpu().numpy().mean()), "p_success_hist": hist.tolist()}


def extra_c5():
    import ctypes
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    n, layers = 20, 50
    res, first = {}, {}
    for dt, B, name in ((qc.QC_C64, 64, "c64_batch64"), (qc.QC_C128, 1, "c128_batch1")):
        circs = W.ansatz(n, layers, seed=5, batch=B)
        P = circs[0].n_params
        gl = []
        for l in range(layers):
            for q in range(n):
                gl.append(qc.Gate(qc.QC_G_RY, q, 0, l * 2 * n + 2 * q))
                gl.append(qc.Gate(qc.QC_G_RZ, q, 0, l * 2 * n + 2 * q + 1))
            for i in range(n):
                gl.append(qc.Gate(qc.QC_G_CNOT, i, (i + 1) % n, 0))
        gates = (qc.Gate * len(gl))(*gl)
        terms = W.ansatz_hamiltonian(n)
        tarr = (qc.PauliTerm * len(terms))(*[qc.PauliTerm(x, z, c) for (x, z, c) in terms])
        theta = torch.tensor(np.stack([c.theta for c in circs]), dtype=torch.float64, device="cuda")
        cdt = torch.complex64 if dt == qc.QC_C64 else torch.complex128
        psi = torch.empty(B << n, dtype=cdt, device="cuda")
        lam = torch.empty_like(psi)
        E = torch.empty(B, dtype=torch.float64, device="cuda")
        grad = torch.empty(B, P, dtype=torch.float64, device="cuda")
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        L = qc.lib()
        vp = ctypes.c_void_p

        def fwd():
            return L.qc_circuit_forward(n, dt, B, gates, len(gl), vp(theta.data_ptr()), P, vp(psi.data_ptr()), s)

        def adj():
            return L.qc_adjoint_grad(n, dt, B, gates, len(gl), vp(theta.data_ptr()), P, P, tarr, len(terms),
                                     vp(psi.data_ptr()), vp(lam.data_ptr()), vp(E.data_ptr()),
                                     vp(grad.data_ptr()), s)
        fwd(); adj()
        torch.cuda.synchronize()
        a, b, c_ = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(); rc1 = fwd(); b.record(); rc2 = adj(); c_.record()
        torch.cuda.synchronize()
        if rc1 or rc2:
            res[name] = {"error": qc.last_error()}
            continue
        tf, tg = a.elapsed_time(b), b.elapsed_time(c_)
        res[name] = {"qubits": n, "gates": len(gl), "angles": P, "batch": B, "forward_ms": tf,
                     "grad_ms (forward+backward)": tg, "grad_time_over_forward": tg / tf,
                     "energy_mean": float(E.mean().item())}
        # batch element 0 has the same angles in both runs (seed 5, row 0)
        fwd()
        torch.cuda.synchronize()
        nrm = float((psi[: 1 << n].abs().double() ** 2).sum().item())
        first[name] = (float(E[0].item()), grad[0].cpu().numpy(), nrm)
    e64, g64, n64 = first["c64_batch64"]
    e128, g128, n128 = first["c128_batch1"]
    res["c64_vs_c128"] = {"energy_abs_diff": abs(e64 - e128), "grad_max_abs_diff": float(np.max(np.abs(g64 - g128))),
                          "grad_max_abs_c128": float(np.max(np.abs(g128))),
                          "norm_error_after_forward_c64": abs(n64 - 1.0), "norm_error_after_forward_c128": abs(n128 - 1.0),
                          "note": "batch element 0 of the complex64 run against the complex128 run, same angles"}
    return res


def extra_f3(n=14, B=64):
    """The paper's multiverse noise and density matrix (sec. 6.1-6.3): B
    Grover runs of n qubits, each noisy universe with one Wigner intrusion
    (D^{1/2} or D^{3/2}) at a random stage, then rho explicitly and its
    spectrum through the Gram matrix (complex128)."""
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    import workloads as W
    k = W.grover_iterations(n)
    m = int(W.marked_indices(W.rng(140), n, 1)[0])
    mv = W.multiverse_noise(B, n, k, seed=14)
    t = torch.empty((B, 1 << n), dtype=torch.complex128, device="cuda")
    ops = {b: {} for b in range(B)}
    for b in range(B):
        if mv.kind[b]:
            twoj = 1 if mv.kind[b] == 1 else 3
            ops[b] = qc.qc_wigner_d(twoj, mv.alpha[b], mv.beta[b], 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(B):
        s = qc.State(n, qc.QC_C128, tensor=t[b])
        s.uniform()
        for it in range(k + 1):
            if mv.kind[b] and it == mv.eloc[b]:
                if mv.kind[b] == 1:
                    s.apply_1q(int(mv.qhit[b]), ops[b])
                else:
                    qc.qc_apply_2q(s.h, int(mv.qhit[b]), int(mv.qhit2[b]), ops[b])
            if it < k:
                s.grover_step([m])
        s.close()
    torch.cuda.synchronize()
    t_runs = time.perf_counter() - t0
    N = 1 << n
    rho = torch.empty(N * N, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    qc.qc_density_matrix(t.data_ptr(), n, qc.QC_C128, B, mv.P, rho.data_ptr(), stream)
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    qc.qc_density_matrix(t.data_ptr(), n, qc.QC_C128, B, mv.P, rho.data_ptr(), stream)
    b_.record()
    torch.cuda.synchronize()
    t_rho = a.elapsed_time(b_)
    p_m = float(rho[m * N + m].real.item())
    del rho
    # the same ensemble in complex64: rho on the tensor cores
    t64 = t.to(torch.complex64)
    rho64 = torch.empty(N * N, dtype=torch.complex64, device="cuda")
    qc.qc_density_matrix(t64.data_ptr(), n, qc.QC_C64, B, mv.P, rho64.data_ptr(), stream)
    a.record()
    for _ in range(3):
        qc.qc_density_matrix(t64.data_ptr(), n, qc.QC_C64, B, mv.P, rho64.data_ptr(), stream)
    b_.record()
    torch.cuda.synchronize()
    t_rho64 = a.elapsed_time(b_) / 3
    rho64_mm = float(rho64[m * N + m].real.item())
    del rho64, t64
    qc.qc_mixed_spectrum(t.data_ptr(), n, qc.QC_C128, B, mv.P)
    t0 = time.perf_counter()
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(t.data_ptr(), n, qc.QC_C128, B, mv.P)
    t_spec = time.perf_counter() - t0
    return {"qubits": n, "universes": B, "grover_iterations": k, "runs_ms": t_runs * 1e3,
            "rho_ms (complex128, 4^n entries)": t_rho, "rho_GB/s_written": N * N * 16 / (t_rho * 1e6),
            "rho_ms (complex64, tensor cores, synchronous call)": t_rho64,
            "rho64_GB/s_written": N * N * 8 / (t_rho64 * 1e6),
            "rho64_tensor_TFLOP/s (bf16 digit products executed)": 2.0 * 8 * (2 * B) * (2 * N * N) / (t_rho64 * 1e9),
            "rho64_mm_minus_rho128_mm": rho64_mm - p_m,
            "spectrum_ms (Gram + Householder/bisection, synchronous)": t_spec * 1e3, "trace": tr, "purity": pur,
            "entropy": ent, "p_success_rho_mm": p_m, "largest_eigenvalue": float(ev[0])}


def extra_dense(n=30, reps=5):
    """The dense k-qubit block on the tensor cores: a random 32 x 32 unitary
    on 5 qubits of an n-qubit complex64 state (tcgen05 kind::f16, bf16 digit
    slices), on the lowest five qubits, on qubits 5..9 and on five scattered
    ones.  Bound: HBM (2S per launch); the tensor work executed is 8 digit
    products x 256 flops per amplitude."""
    import json as _json
    import numpy as np
    import torch
    import paper_0902_0699_gb300 as qc
    g = np.random.default_rng(5)
    A = g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))
    U, _ = np.linalg.qr(A)
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    res = {}
    s = qc.State(n, qc.QC_C64)
    s.uniform()
    for name, qs in (("qubits_0_4", [0, 1, 2, 3, 4]), ("qubits_5_9", [5, 6, 7, 8, 9]),
                     ("scattered", [n - 5, 3, n - 13, 9, n - 1])):
        qc.qc_apply_dense(s.h, qs, U)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            qc.qc_apply_dense(s.h, qs, U)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        S = (1 << n) * 8
        gbs = 2 * S / ms / 1e6
        tflops = 8 * 256 * (1 << n) / ms / 1e9
        res[name] = {"qubits": qs, "ms": ms, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm,
                     "tensor_TFLOP/s (bf16 executed)": tflops, "frac_of_bf16_peak": tflops / bf16}
    s.close()
    res["note"] = ("per launch: %d-qubit complex64, one tile of 128 groups per MMA round (tcgen05 kind::f16 bf16, "
                   "M128 N64 K64 x 8 digit products = 32 MMAs of K16); bf16 peak = measured %.0f TFLOP/s" % (n, bf16))
    return res


# ------------------------------------------------------------ CPU oracle ----

def cpu_oracle_sample(n=22, iters=2):
    """The oracle as it stands on the host cores: HALL, `iters` literal
    Grover operators, the literal QFT and the gate sweep, on an n-qubit
    complex128 state.  Returns (amp-updates/s with the same operator count
    as the GPU step, seconds, threads)."""
    import numpy as np
    import oracle as O
    import workloads as W
    O.set_threads(os.cpu_count() or 1)
    N = 1 << n
    psi = O.zero_state(n)
    marked = W.marked_indices(W.rng(2026), n, 8)
    t0 = time.perf_counter()
    O.hall(psi, n)
    for _ in range(iters):
        O.grover_step(psi, n, marked)
    O.qft(psi, n)
    p = O.probs(psi, n)
    O.sample_from_probs(p, 12345, 1000)
    for t in range(n):
        O.apply_1q(psi, n, t, O.H_MAT)
        O.cnot(psi, n, (t + 1) % n, t)
        O.cphase(psi, n, (t + 1) % n, t, 1)
    el = time.perf_counter() - t0
    ops = 1 + iters + 1 + 3 * n
    return ops * N / el, el, O.get_threads(), ops


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    n_s = 25
    vals, secs = [], []
    for _ in range(args.warmup):
        cpu_oracle_sample(n_s, 1)
    for _ in range(args.steps):
        v, el, cores, ops = cpu_oracle_sample(n_s, 3)
        vals.append(v)
        secs.append(el)
    value = statistics.mean(vals)
    sample = "per step: %d-qubit complex128 HALL, 3 literal Grover operators (8 marked), literal QFT, probs + 1000 samples, H/CNOT/CPHASE sweep over all t (%d operators)" % (n_s, ops)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "grover%d_qft_sweep_c128" % args.n, "qubits": args.n,
                       "reference_sample_qubits": n_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ main ----

def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    import torch
    import torch.distributed as dist
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.only:
        fn = {"c64": extra_c64, "c1": extra_c1, "c2": extra_c2, "c4": extra_c4, "c5": extra_c5,
              # a small trajectory batch (96 instances, 16..18 qubits) for profiling
              "c4s": lambda: extra_c4(96, 16, 18, seed=7, autotune=0), "f3": extra_f3,
              "dense": extra_dense, "dense26": lambda: extra_dense(26, 2), "red": extra_red,
              "u2": extra_u2_sweep, "u2_26": lambda: extra_u2_sweep(26), "rho64": extra_rho64}[args.only]
        print(json.dumps({args.only: fn()}), flush=True)
        return 0
    out, st, step_fn, ops, N = run_ours(args, ws, rank, local)
    if not args.no_e2e:
        try:
            out["e2e"] = run_e2e(args, st, step_fn, ops, N)
        except Exception as e:  # report, do not hide
            out["e2e"] = {"error": repr(e)}
    st.close()
    del st
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu:
        v, el, cores, nops = cpu_oracle_sample(25, 3)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "25-qubit complex128: HALL, 3 literal Grover operators, literal QFT, probs + 1000 samples, H/CNOT/CPHASE sweep (%d operators, %.1f s)" % (nops, el)}
    if rank == 0 and not args.no_extras:
        extras = {}
        for name, fn in (("c64_n32", extra_c64), ("u2_sweep_n30_c128", extra_u2_sweep),
                         ("grover_n10", extra_c1), ("random_n24", extra_c2),
                         ("trajectories_4096", extra_c4), ("adjoint_n20", extra_c5),
                         ("multiverse_density_n14", extra_f3), ("dense_block_k5_n30_c64", extra_dense)):
            try:
                extras[name] = fn()
            except Exception as e:
                extras[name] = {"error": repr(e)}
            torch.cuda.empty_cache()
        out["extras"] = extras
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
