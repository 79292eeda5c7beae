"""Benchmark of the lq2d solver: PCG iterations/s and time-to-solve at a
1e-8 relative KKT residual, on the K = N = 256, n = 4, m = 2, T = 200
synthetic grid (52.7 M multipliers, S = L = 2, FP64), the largest
single-GPU workload; the K = N = 64, T = 100 grid is measured beside it with
the same protocol.

One step = one full pass of the method over the resident problem: the setup
(inverses, splitting blocks, banded block-Cholesky factors of Phi_bar), the
PCG solve to the tolerance (Algorithm 1 with Algorithm 2 as
preconditioner), and the recovery of x, u and the KKT residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica (the method has no data-path exchange on one GPU); value is the sum
of iterations over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_04980_gb300 import synth  # noqa: E402

METRIC = "PCG iters/s (time-to-solve at 1e-8 rel KKT residual)"
UNIT = "iters/s"
# FP64 peak of the GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 flops x
# 2.07 GHz (the nominal 1.25 TFLOP/s expressed in unit counts and clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="grid256_T200", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--also", default="grid64_T100",
                    help="second workload measured with the same protocol (FP64, modes 1 and 2, roofline) and "
                         "reported under its own key; 'none' to skip")
    ap.add_argument("--aux-steps", type=int, default=5,
                    help="steps of the passes beside the timed region (per-launch timing, precision comparison, "
                         "end to end), at most --steps")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--driver", choices=["graph", "stream"], default="graph")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed2"], default="fp64",
                    help="fp64: FP64 everywhere; mixed: FP32 preconditioner, FP64 residual/dots/updates; "
                         "mixed2: also the product Delta d in FP32, with FP64 residual replacement per phase")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the timed mixed-precision comparison on the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-threads", type=int, default=0, help="set LQ2D_OPT_SWEEP_THREADS (0: library default)")
    ap.add_argument("--sweep-steps", type=int, default=-1,
                    help="set LQ2D_OPT_SWEEP_STEPS, time steps per lane of the n = 4 FP32 sweeps (-1: default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default FP32 sweep schedule in the precision comparison")
    ap.add_argument("--cpu-iters", type=int, default=3, help="oracle PCG steps in the all-cores CPU sample")
    ap.add_argument("--cpu-iters-one", type=int, default=1, help="oracle PCG steps in the one-thread CPU sample")
    ap.add_argument("--batch", type=int, default=0,
                    help="time the batched solve of this many uneven instances (K, N in 8..64, T in 50..200) "
                         "against solving them one after another")
    ap.add_argument("--warmstart", type=int, default=0,
                    help="learned warm start: train the network on this many solver-generated instances of the "
                         "K = N = 128, T = 100 family, then time held-out solves from its guess and from zero")
    ap.add_argument("--ws-steps", type=int, default=1500, help="training steps of the warm-start network")
    ap.add_argument("--ws-eval", type=int, default=50, help="held-out instances (seeds 100000+) evaluated")
    ap.add_argument("--ws-buffer", type=int, default=2048,
                    help="training pairs kept on the device; with more --warmstart instances than this the "
                         "network trains online (pairs generated group by group into a ring buffer)")
    ap.add_argument("--ws-group", type=int, default=32,
                    help="training pairs per multi-right-hand-side solve (seeds sharing one coupling value); "
                         "1 = one mixed-precision solve per pair")
    ap.add_argument("--multirhs", type=int, default=0,
                    help="multi-right-hand-side solve: this many instances of the batch family (K, N in 8..64, "
                         "T in 50..200), each with 32 initial states x0 ~ N(0, 1), against single solves")
    ap.add_argument("--mrhs-apply", type=int, default=0,
                    help="apply the 32-right-hand-side tensor-core preconditioner (S = L = 2) this many times on "
                         "--workload and print its time per application (the launch sequence profiled for the "
                         "multi-right-hand-side sweep)")
    return ap.parse_args()


# --------------------------------------------------------------------------
# distributed helpers (replicas; the barrier and max are timing only)
# --------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def reduce(self, value, op):
        if self.pg is None:
            return value
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64,
                         device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------
# clock sampling during the timed region
# --------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return self.parse(lines)

    @classmethod
    def parse(cls, lines):
        """Median SM clock, maximum clock and the throttle reasons seen in
        nvidia-smi's CSV samples (the FIELDS columns, no header, no units);
        None without a usable sample."""
        sm, mx, reasons = [], [], set()
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(cls.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic flop model of one NBJM sweep (FP64 path)
# --------------------------------------------------------------------------

def band_solve_flops(K, n, cols):
    """Forward plus backward substitution with the banded block-Cholesky
    factor of one Phi_bar_{v,t} block (Section IV-B), envelope entries only:
    each multiply-add counts 2 flops, each diagonal scaling 1.  This is the
    algorithmic count whatever form the kernel stores the factor in; the
    sweeps' unit-factor form (dense F2, F1, N1 and D^-1 blocks, the
    block-diagonal coupling E in the backward step) executes as many
    multiply-adds per interior pair-row."""
    f = 0
    for i in range(K):
        for a in range(cols * n):
            e = a
            if i >= 1:
                e += cols * n
            if i >= 2:
                e += (2 * n if a < n else n) if cols == 2 else n
            f += 2 * e + 1
    return 2 * f


def sweep_kernel_name(sched, vt):
    """The sweep kernel a schedule runs: the bulk-copy FP32 kernel (n = 4,
    steps per lane >= 1), the two-ended tiled kernel, or the tiled kernel."""
    if vt == "float" and sched.get("steps_per_lane", 0) >= 1:
        return "nbjm_sweep_bulk_kernel<*,%d,%d>" % (sched["steps_per_lane"], sched["threads"])
    if sched.get("two_ended"):
        return "nbjm_sweep_twisted_kernel<4,*,%s,%d>" % (vt, sched["threads"])
    return "nbjm_sweep_kernel<4,*,%s,%d>" % (vt, sched["threads"])


def sweep_flops(g: synth.GridLQ):
    """Algorithmic flops of one sweep launch of each kind, keyed by variant."""
    K, N, T, n = g.K, g.N, g.T, g.n
    V = (N + 1) // 2
    pairs_two = N // 2
    pairs_one = V - pairs_two
    band = T * (pairs_two * band_solve_flops(K, n, 2) + pairs_one * band_solve_flops(K, n, 1))
    t0 = K * N * 2 * n * n                      # theta_0 = Q tau, node by node
    # valid neighbour counts
    offpair = 0
    nbrs = 0
    for i in range(K):
        for j in range(N):
            s = 1 if (j % 2) else -1
            cand = [(i, j + s), (i - 1, j + s), (i + 1, j + s), (i, j + 2 * s), (i, j - 2 * s)]
            offpair += sum(0 <= a < K and 0 <= b < N for a, b in cand)
            nbrs += 1 + sum(0 <= a < K and 0 <= b < N for a, b in ((i, j - 1), (i, j + 1), (i - 1, j), (i + 1, j)))
    omega = T * offpair * 2 * n * n
    xi = 2 * T * nbrs * 2 * n * n               # A Q^-1 delta_{t-1} for t >= 1, Q^-1 A' delta_{t+1} for t < T
    unknowns = K * N * (T + 1) * n
    return {
        "update": band + t0 + 6 * unknowns,
        "omega": band + t0 + omega,
        "omega_mu": band + t0 + omega + 2 * unknowns,
        "xi": band + t0 + xi,
        "plain": band + t0,
    }


# Algorithmic bytes per unknown of each FP32 sweep of the mixed mode: every
# vector operand read once and every result written once (r, delta, y, d and
# r_theta are FP64; theta and delta^(s) FP32); factors and node blocks are
# time-invariant, L2-resident and amortised over the T+1 time slices.
MIXED_SWEEP_BYTES = {"update": 4 * 8 + 2 * 8 + 4, "omega": 8 + 4 + 4, "xi": 8 + 4 + 8 + 4,
                     "omega_mu": 8 + 4 + 4 + 8 + 8}


def sweep_bytes_of_solve(g, iterations):
    unknowns = g.nodes * (g.T + 1) * g.n
    full = sum(MIXED_SWEEP_BYTES.values()) * unknowns
    return max(iterations - 1, 0) * full + (MIXED_SWEEP_BYTES["update"] * unknowns if iterations > 0 else 0)


def sweep_flops_of_solve(fl, iterations, S=2, L=2):
    """Flops of the sweep launches timed in one solve: every PCG step but the
    last runs update, omega, xi, omega_mu (S = L = 2); the last one stops
    after the update sweep."""
    assert S == 2 and L == 2
    full = fl["update"] + fl["omega"] + fl["xi"] + fl["omega_mu"]
    return max(iterations - 1, 0) * full + (fl["update"] if iterations > 0 else 0)


def measured_hbm_gbs():
    """The measured copy bandwidth of the GB300s (GB/s), else
    the profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


KERNEL_SOURCES = {
    "fp64": ("sweep_tiled.cuh", "common.cuh", "kernels.h"),
    "fp32": ("sweep_bulk.cuh", "sweep_bulk.cu", "sweep_tiled.cuh", "common.cuh", "kernels.h"),
}


def kernel_source_hash(precision="fp64"):
    """Hash of the sources of the sweep kernels of one precision (the FP64
    tiled sweep; the FP32 bulk-copy and tiled sweeps)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[precision]:
        h.update(open(os.path.join(ROOT, "paper_2304_04980_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, precision="fp64", kernel=None):
    """DRAM bytes per sweep launch from the committed ncu summary of that
    workload and sweep precision, if it was taken on the current kernel
    source and, where the summary names its kernel, on `kernel` (else
    None)."""
    name = "nbjm_sweep_%s.md" % workload if precision == "fp64" else "nbjm_sweep_f32_%s.md" % workload
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel source hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram bytes per launch \(read\+write\):\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(precision):
        return None
    m_kernel = re.search(r"profiled kernel:\s*(\S+)", text)
    if kernel is not None and m_kernel and m_kernel.group(1) != kernel:
        return None
    return float(m_bytes.group(1))


# --------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, single-threaded, bounded sample
# --------------------------------------------------------------------------

def host_cores():
    """Cores this process may run on, and how many oracle worker processes
    the host's free memory allows (each holds about 1.5 GB of splitting
    blocks at the 256 x 256 x 200 size)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    try:
        avail_gb = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 1e9
    except (ValueError, OSError):
        avail_gb = 1e9
    return cores, max(1, min(cores, int(avail_gb / 3.0)))


CPU_SCRIPT = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
from oracle import lq2d_oracle as O
from oracle import slab_pcg as SP
from paper_2304_04980_gb300 import synth


def main():
    g = synth.workload(%(workload)r)
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    t0 = time.perf_counter()
    so = SP.SlabOracle(P, workers=%(workers)d)
    t1 = time.perf_counter()
    clock = []
    so.solve(1e-300, 2, 2, %(iters)d, confirm_true_residual=False, step_clock=clock)
    so.close()
    print(json.dumps({"setup_s": t1 - t0, "iters": len(clock) - 1, "loop_s": clock[-1] - clock[0],
                      "clock": clock}))


if __name__ == "__main__":
    main()
"""


def run_oracle_steps(workload, workers, iters, timeout=1800):
    """The oracle's Algorithm 1 loop (slab form, S = L = 2) for `iters`
    passes on the full workload, in a subprocess with `workers` processes
    and one BLAS thread each; returns the parsed timing record or a failure
    string."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = CPU_SCRIPT % {"root": ROOT, "workload": workload, "iters": iters, "workers": workers}
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        tail = out.stderr.strip().splitlines()[-1][:200] if out.stderr.strip() else "exit %d" % out.returncode
        return "failed: " + tail
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(workload, iters_all, iters_one):
    """The oracle timed on the host: on all cores this process may use
    (the slabs split over worker processes), and on one thread."""
    cores, workers = host_cores()
    res = {"unit": UNIT, "kind": "oracle"}
    r = run_oracle_steps(workload, workers, iters_all)
    if isinstance(r, str):
        res.update({"value": None, "cores": workers, "sample": r})
    else:
        res.update({"value": r["iters"] / r["loop_s"], "cores": workers, "host_cores": cores,
                    "sample": "%d PCG steps (Algorithm 1 loop, S = L = 2, every step timed after the initial "
                              "residual and preconditioner) of the slab-by-slab oracle on the full %s problem, "
                              "%d worker processes splitting the time slabs, one BLAS thread each; oracle "
                              "setup (blocks, splitting, banded Cholesky per column pair) %.1f s not counted"
                              % (r["iters"], workload, workers, r["setup_s"]),
                    "setup_s": r["setup_s"], "loop_s": r["loop_s"]})
    r1 = run_oracle_steps(workload, 1, iters_one)
    if isinstance(r1, str):
        res["single_thread"] = {"value": None, "cores": 1, "sample": r1}
    else:
        res["single_thread"] = {
            "value": r1["iters"] / r1["loop_s"], "unit": UNIT, "cores": 1,
            "sample": "%d PCG step(s) of the same oracle on the full %s problem, one process, one BLAS thread; "
                      "setup %.1f s not counted" % (r1["iters"], workload, r1["setup_s"]),
            "setup_s": r1["setup_s"], "loop_s": r1["loop_s"]}
    return res


# --------------------------------------------------------------------------
# reference arm: the oracle timed on the host cores
# --------------------------------------------------------------------------

def run_reference(args, dist):
    """The paper ships no code, so the reference arm is the CPU oracle as it
    stands (slab form), on all host cores, on this arm's workload: one
    Algorithm 1 loop of W + K passes, the last K timed step by step."""
    if dist.rank != 0:
        return
    cores, workers = host_cores()
    g = synth.workload(args.workload)
    r = run_oracle_steps(args.workload, workers, args.warmup + args.steps, timeout=3600)
    if isinstance(r, str):
        print(json.dumps({"impl": "reference", "unavailable": "oracle run " + r}), flush=True)
        return
    clock = r["clock"]
    t_steps = clock[args.warmup + args.steps] - clock[args.warmup]
    value = args.steps / t_steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_steps * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "K": g.K, "N": g.N, "T": g.T, "n": g.n, "m": g.m, "S": 2, "L": 2,
                   "tol": args.tol, "precision": "fp64", "driver": "cpu oracle",
                   "l2": "not applicable (host)", "parallelism": "%d host processes" % workers},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "host_cores": cores, "kind": "oracle",
                         "sample": "each step = one PCG step (Algorithm 1 loop pass, S = L = 2) of the slab-by-slab "
                                   "CPU oracle (numpy/scipy, as it stands) on the full problem, %d worker "
                                   "processes; oracle setup %.1f s and the initial residual not timed"
                                   % (workers, r["setup_s"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args, dist):
    import torch

    from paper_2304_04980_gb300 import lq2d

    lq2d.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    aux = max(1, min(args.aux_steps, args.steps))

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None

    def measure(workload, headline):
        """The protocol on one workload: the timed region (K steps, device
        events, L2 flushed before each), the per-launch roofline pass, the
        precision comparison and, for the headline, the end-to-end pass."""
        g = synth.workload(workload)
        host = [np.ascontiguousarray(a) for a in g.arrays()]
        inputs = [torch.from_numpy(a).to(dev) for a in host]
        prob = lq2d.Problem.from_device(g.K, g.N, g.T, g.n, g.m, *inputs, stream=stream)
        if args.precision != "fp64":
            prob.set_precision(1 if args.precision == "mixed" else 2)
        if args.driver == "stream":
            prob.set_option(lq2d.OPT_DRIVER, 1)
        if args.sweep_threads:
            prob.set_option(lq2d.OPT_SWEEP_THREADS, args.sweep_threads)
        if args.sweep_steps >= 0:
            prob.set_option(lq2d.OPT_SWEEP_STEPS, args.sweep_steps)
        x = torch.empty((g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
        u = torch.empty((g.T, g.nodes, g.m), dtype=torch.float64, device=dev)
        lam = torch.empty_like(x)
        max_iter = 100000

        def step():
            prob.update_device(*inputs, stream=stream)
            return prob.solve_device(args.tol, 2, 2, max_iter, x=x, u=u, costate=lam, stream=stream)

        def timed(nsteps):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(nsteps)]
            its, rls = [], []
            for k in range(nsteps):
                flush.zero_()
                evs[k][0].record(stream)
                out = step()
                evs[k][1].record(stream)
                its.append(out["iterations"])
                rls.append(out["rel_kkt"])
            torch.cuda.synchronize()
            return [a.elapsed_time(b) for a, b in evs], its, rls

        # the library's autotuner picks the sweep schedule of this precision
        # for the shape (outside the timed region, as a user would at set-up)
        tuned = None
        if not args.no_autotune and not (args.sweep_threads or args.sweep_steps >= 0):
            tuned = prob.autotune(2, 2, 3, stream=stream)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()

        # ---- timed region
        res = {"g": g}
        clocks = Clocks(uuid) if headline else None
        launches0 = prob.stats()["launches_total"]
        if clocks:
            clocks.start()
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        step_ms, iters, rels = timed(args.steps)
        dist.barrier()
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        res["clocks"] = clocks.stop() if clocks else None
        stt = prob.stats()
        res["schedule"] = {"threads": stt["sweep_threads"], "steps_per_lane": stt["sweep_steps"],
                           "two_ended": int(prob.get_option(lq2d.OPT_TWISTED)), "autotuned": tuned is not None}
        res["launches"] = prob.stats()["launches_total"] - launches0
        res["dev_ms"] = sum(step_ms)
        res["iters"] = iters
        res["rels"] = rels
        res["wall_ms"] = (w1 - w0) * 1e3

        # ---- roofline of the dominant kernel (NBJM sweep): per-launch events
        # on the solve stream, over `aux` steps run again with timing on
        prob.set_option(lq2d.OPT_TIMING, 1)
        sweep_ms, sweep_launches, delta_ms, delta_launches, fl_total, by_total = 0.0, 0, 0.0, 0, 0, 0
        fl = sweep_flops(g)
        for _ in range(aux):
            flush.zero_()
            out = step()
            st = prob.stats()
            sweep_ms += st["sweep_ms"]
            sweep_launches += st["sweep_launches"]
            delta_ms += st["delta_ms"]
            delta_launches += st["delta_launches"]
            fl_total += sweep_flops_of_solve(fl, out["iterations"])
            by_total += sweep_bytes_of_solve(g, out["iterations"])
        prob.set_option(lq2d.OPT_TIMING, 0)
        measured_note = ("CUDA events around each sweep launch on the solve stream, a second pass over %d steps "
                         "of the same workload" % aux)
        if args.precision == "fp64":
            achieved = fl_total / (sweep_ms / 1e3) / 1e12
            res["roofline"] = {
                "kernel": sweep_kernel_name(res["schedule"], "double"), "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": profiled_traffic(workload, "fp64", sweep_kernel_name(res["schedule"], "double")),
                "avg_launch_ms": sweep_ms / max(sweep_launches, 1), "launches_timed": sweep_launches,
                "flops_per_launch": fl_total / max(sweep_launches, 1),
                "peak_note": "FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)",
                "measured": measured_note,
                "delta_apply_ms_per_launch": delta_ms / max(delta_launches, 1),
            }
        else:
            peak = measured_hbm_gbs()
            achieved = by_total / (sweep_ms / 1e3) / 1e9
            res["roofline"] = {
                "kernel": sweep_kernel_name(res["schedule"], "float"), "bound": "hbm", "achieved": achieved,
                "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(workload, "fp32", sweep_kernel_name(res["schedule"], "float")),
                "avg_launch_ms": sweep_ms / max(sweep_launches, 1), "launches_timed": sweep_launches,
                "bytes_per_launch": by_total / max(sweep_launches, 1),
                "fp32_tflops": fl_total / (sweep_ms / 1e3) / 1e12,
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "measured": measured_note,
                "delta_apply_ms_per_launch": delta_ms / max(delta_launches, 1),
            }

        # ---- the same workload in the other precisions, same protocol; the
        # FP32 sweep's roofline (bytes against the copy bandwidth) beside it
        compare = None
        if not args.no_compare and args.precision == "fp64":
            compare = []
            for mode, label in ((1, "mixed: FP32 preconditioner, FP64 residual/dots/updates"),
                                (2, "mixed2: FP32 preconditioner and Delta product, FP64 residual replacement")):
                prob.set_precision(mode)
                # the library's autotuner picks the FP32 sweep schedule for this
                # shape (outside the timed region, as a user would at set-up)
                tuned = (prob.autotune(2, 2, 3, stream=stream)
                         if not args.no_autotune and not (args.sweep_threads or args.sweep_steps >= 0) else None)
                for _ in range(args.warmup):
                    step()
                c_ms, c_its, c_rels = timed(aux)
                c_dev = sum(c_ms)
                stt = prob.stats()
                entry = {"precision": label, "value": sum(c_its) / (c_dev / 1e3), "unit": UNIT,
                         "ms_per_step": c_dev / aux, "steps": aux,
                         "sweep_schedule": {"threads": stt["sweep_threads"], "steps_per_lane": stt["sweep_steps"],
                                            "two_ended": int(prob.get_option(lq2d.OPT_TWISTED)),
                                            "autotuned": tuned is not None},
                         "iterations_per_solve": sum(c_its) / len(c_its), "rel_kkt_residual": max(c_rels),
                         "speedup_time_to_solve": (res["dev_ms"] / args.steps) / (c_dev / aux)}
                prob.set_option(lq2d.OPT_TIMING, 1)
                s_ms, s_n, b_tot = 0.0, 0, 0
                for _ in range(min(aux, 3)):
                    flush.zero_()
                    out = step()
                    st = prob.stats()
                    s_ms += st["sweep_ms"]
                    s_n += st["sweep_launches"]
                    b_tot += sweep_bytes_of_solve(g, out["iterations"])
                prob.set_option(lq2d.OPT_TIMING, 0)
                peak = measured_hbm_gbs()
                ach = b_tot / (s_ms / 1e3) / 1e9
                entry["sweep_roofline"] = {"kernel": sweep_kernel_name(entry["sweep_schedule"], "float"),
                                           "bound": "hbm",
                                           "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                           "traffic": profiled_traffic(workload, "fp32", sweep_kernel_name(
                                               entry["sweep_schedule"], "float")),
                                           "avg_launch_ms": s_ms / max(s_n, 1),
                                           "bytes_per_launch": b_tot / max(s_n, 1)}
                compare.append(entry)
            prob.set_precision(0)
        res["compare"] = compare

        # ---- end to end: host (pinned) inputs in, host outputs back, per step
        if headline:
            pinned = [torch.from_numpy(a).pin_memory() for a in host]
            # the outputs land in pinned host buffers too (a user's numpy views of them)
            outs = [torch.empty(shape, dtype=torch.float64).pin_memory()
                    for shape in ((g.T + 1, g.nodes, g.n), (g.T, g.nodes, g.m), (g.T + 1, g.nodes, g.n))]
            xh, uh, lh = (o.numpy() for o in outs)
            res["h2d"] = sum(a.nbytes for a in host)
            res["d2h"] = xh.nbytes + uh.nbytes + lh.nbytes
            torch.cuda.synchronize()
            e_iters = 0
            e0 = time.perf_counter()
            for _ in range(aux):
                flush.zero_()
                torch.cuda.synchronize()
                prob.update(*[p.data_ptr() for p in pinned])
                out = prob.solve(args.tol, 2, 2, max_iter, out=(xh, uh, lh))
                e_iters += out["iterations"]
            e1 = time.perf_counter()
            res["e2e_value"] = dist.reduce(e_iters, "sum") / dist.reduce(e1 - e0, "max")
            res["e2e_steps"] = aux
        prob.close()
        del inputs, x, u, lam
        torch.cuda.empty_cache()
        return res

    main = measure(args.workload, True)
    g = main["g"]
    tot_iters = sum(main["iters"])
    all_iters = dist.reduce(tot_iters, "sum")
    max_ms = dist.reduce(main["dev_ms"], "max")
    value = all_iters / (max_ms / 1e3)

    second = None
    if args.also and args.also != "none" and args.also != args.workload:
        o = measure(args.also, False)
        og = o["g"]
        second = {"workload": args.also, "K": og.K, "N": og.N, "T": og.T, "n": og.n, "m": og.m,
                  "value": sum(o["iters"]) / (o["dev_ms"] / 1e3), "unit": UNIT, "steps": args.steps,
                  "time_to_solve_ms": o["dev_ms"] / args.steps,
                  "iterations_per_solve": sum(o["iters"]) / len(o["iters"]), "rel_kkt_residual": max(o["rels"]),
                  "roofline": o["roofline"], "sweep_schedule": o["schedule"], "compare_precision": o["compare"]}

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_iters, args.cpu_iters_one)

    if dist.rank == 0:
        mean_iters = tot_iters / len(main["iters"])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["dev_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "K": g.K, "N": g.N, "T": g.T, "n": g.n, "m": g.m, "S": 2,
                       "L": 2, "tol": args.tol, "precision": args.precision, "driver": args.driver,
                       "l2": "flushed before each step (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if dist.world > 1 else "single"},
            "time_to_solve_ms": main["dev_ms"] / args.steps,
            "iterations_per_solve": mean_iters,
            "rel_kkt_residual": max(main["rels"]),
            "wall_ms": main["wall_ms"],
            "roofline": main["roofline"],
            "sweep_schedule": main["schedule"],
            "compare_precision": main["compare"],
            "also": second,
            "cpu_baseline": cpu,
            "e2e": {"value": main["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": main["h2d"],
                    "d2h_bytes_per_step": main["d2h"], "steps": main["e2e_steps"]},
            "clocks": main["clocks"],
            "gpu_launches": main["launches"],
        }
        print(json.dumps(line), flush=True)


def run_batch(args, dist):
    """Batched workload: `args.batch` uneven instances solved by one graph
    launch, against the same instances solved one after another."""
    import torch

    from paper_2304_04980_gb300 import lq2d

    lq2d.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    grids = synth.batch_grids(args.batch)
    probs = [lq2d.Problem.from_grid(gr) for gr in grids]
    if args.precision != "fp64":
        for p in probs:
            p.set_precision(1 if args.precision == "mixed" else 2)
    batch = lq2d.Batch(probs)
    unknowns = sum(gr.nodes * (gr.T + 1) * gr.n for gr in grids)
    tuned = None
    if args.precision == "fp64":
        tuned = batch.autotune(2, 2, 3, stream=stream)
    for _ in range(args.warmup):
        batch.solve(args.tol, 2, 2, 100000, stream=stream)
    torch.cuda.synchronize()
    persistent = batch.get_option(lq2d.BATCH_USES_PERSISTENT)

    def timed_batch(nsteps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        its = 0
        for k in range(nsteps):
            ev[k][0].record(stream)
            out = batch.solve(args.tol, 2, 2, 100000, stream=stream)
            ev[k][1].record(stream)
            its += sum(out["iterations"])
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), its

    launches0 = sum(p.stats()["launches_total"] for p in probs)
    b_ms, its = timed_batch(args.steps)
    launches = sum(p.stats()["launches_total"] for p in probs) - launches0
    # the same batch as one chain per problem in the graph (no persistent loop)
    chains = None
    if persistent:
        batch.set_option(lq2d.BATCH_PERSISTENT, 0)
        batch.solve(args.tol, 2, 2, 100000, stream=stream)
        c_ms, _ = timed_batch(max(1, min(args.steps, 2)))
        chains = {"ms_per_solve": c_ms / max(1, min(args.steps, 2)),
                  "speedup_persistent_vs_chains": (c_ms / max(1, min(args.steps, 2))) / (b_ms / args.steps)}
        batch.set_option(lq2d.BATCH_PERSISTENT, 1)
        if tuned is not None:
            batch.set_option(lq2d.BATCH_THREADS, tuned[0])
    # the same instances one after another (one graph launch each; every
    # problem's own graph is built by an untimed solve first)
    for p in probs:
        p.solve_device(args.tol, 2, 2, 100000, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_its = 0
    for p in probs:
        s_its += p.solve_device(args.tol, 2, 2, 100000, stream=stream)["iterations"]
    e1.record(stream)
    torch.cuda.synchronize()
    s_ms = e0.elapsed_time(e1)
    line = {
        "metric": "batched time-to-solve at 1e-8 rel KKT residual (instances/s)", "value": args.steps * len(probs) / (b_ms / 1e3),
        "unit": "instances/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": b_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": "batch%d: K, N in 8..64, T in 50..200, n = 4, m = 2, coupling in 0.02..0.2" % len(probs),
                   "precision": args.precision, "tol": args.tol, "S": 2, "L": 2, "unknowns": unknowns},
        "pcg_iters_per_s": its / (b_ms / 1e3),
        "persistent_loop": bool(persistent),
        "autotuned_threads": None if tuned is None else tuned[0],
        "autotune_dsr_ms": None if tuned is None else tuned[1],
        "chains": chains,
        "sequential": {"ms_for_all": s_ms, "instances_per_s": len(probs) / (s_ms / 1e3), "iterations": s_its},
        "speedup_vs_sequential": s_ms / (b_ms / args.steps),
        "gpu_launches": launches,
    }
    batch.close()
    print(json.dumps(line), flush=True)


def conv_flops_per_sample(sizes, K, N):
    """Multiply-adds x 2 of one forward pass of the 3x3 conv stack."""
    return sum(2.0 * 9 * ci * co * K * N for ci, co in zip(sizes[:-1], sizes[1:]))


def run_warmstart(args, dist):
    """Learned warm start (K = N = 128, n = 4, m = 2, T = 100): training pairs
    from the mixed-precision solver, Adam on the GPU, then held-out solves
    to the tolerance from the network's guess and from zero (FP64 solver)."""
    import torch

    from paper_2304_04980_gb300 import lq2d, warmstart

    lq2d.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    fam = synth.warmstart_family()
    ws = warmstart.WarmStart(fam, channels=64, layers=6, batch=8, seed=0, device=str(dev))
    seeds = range(1000, 1000 + args.warmstart)
    online = args.warmstart > args.ws_buffer
    if online:
        # output scale from the first group; then pairs are generated group
        # by group while the network trains
        ws.generate_grouped(seeds[:args.ws_group], tol=1e-6, group=args.ws_group)
    elif args.ws_group > 1:
        gen_s = ws.generate_grouped(seeds, tol=1e-6, group=args.ws_group)
    else:
        gen_s = ws.generate(seeds, tol=1e-6, precision=1)
    sigma = float(ws.targets.std())
    ws.net.close()
    ws.net = lq2d.WarmStartNet(fam.K, fam.N, fam.T, fam.n, 64, 6, 8, sigma)
    ws.net.set_params(synth.warmstart_init(ws.net.layer_sizes(), 0, 0.1))
    torch.cuda.synchronize()
    if online:
        groups = (args.warmstart + args.ws_group - 1) // args.ws_group
        per_group = max(1, -(-args.ws_steps // groups))
        losses, gen_s, train_s, _ = ws.fit_online(seeds, per_group, tol=1e-6, group=args.ws_group,
                                                  buffer=args.ws_buffer, lr=1e-3, lr_final=5e-5)
        args.ws_steps = per_group * groups
    else:
        t0 = time.perf_counter()
        losses = ws.fit(args.ws_steps, lr=1e-3, lr_final=5e-5)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
    fl = conv_flops_per_sample(ws.net.layer_sizes(), fam.K, fam.N)
    train_tflops = 3.0 * fl * 8 * args.ws_steps / train_s / 1e12
    # warm-up of every path, then the held-out instances: zero and learned
    # starts, each with the FP64 and the mixed-precision solver
    combos = [("zero", False, 0), ("warm", True, 0), ("zero_mixed", False, 1), ("warm_mixed", True, 1)]
    for _, warm, prec in combos:
        ws.solve(99999, tol=args.tol, warm=warm, precision=prec)
    its = {k: [] for k, _, _ in combos}
    secs = {k: [] for k, _, _ in combos}
    errs, guess_errs = [], []
    for seed in range(100000, 100000 + args.ws_eval):
        c, x0 = fam.instance_params(seed)
        guess = ws.guess(c, torch.from_numpy(x0).to(dev))
        ref = None
        for key, warm, prec in combos:
            r = ws.solve(seed, tol=args.tol, warm=warm, precision=prec)
            its[key].append(r["iterations"])
            secs[key].append(r["seconds"])
            if ref is None:
                ref = r["costate"]
                guess_errs.append(float(torch.linalg.norm(guess - ref) / torch.linalg.norm(ref)))
            else:
                errs.append(float(torch.linalg.norm(r["costate"] - ref) / torch.linalg.norm(ref)))
    zero_it, warm_it, zero_s, warm_s = its["zero"], its["warm"], secs["zero"], secs["warm"]
    x0 = torch.from_numpy(fam.instance_params(100000)[1]).to(dev)
    ws.guess(0.1, x0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        ws.guess(0.1, x0)
    e1.record()
    torch.cuda.synchronize()
    guess_ms = e0.elapsed_time(e1) / 10
    zero_ms = 1e3 * float(np.mean(zero_s))
    warm_ms = 1e3 * float(np.mean(warm_s))
    line = {
        "metric": "time-to-solve at 1e-8 rel KKT residual, learned warm start (ms)", "value": warm_ms, "unit": "ms",
        "n_gpus": 1, "steps": args.ws_eval, "warmup": 2, "ms_per_step": warm_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 solve, bf16 weights / f32 net", "data": "synthetic",
        "config": {"workload": "warmstart K = N = 128, n = 4, m = 2, T = 100, coupling 0.02..0.2, x0 ~ N(0, 1)",
                   "train_instances": args.warmstart, "train_steps": args.ws_steps, "batch": 8,
                   "train_generation": ("multi-right-hand-side solves at tol 1e-6, %d seeds per coupling value"
                                        % args.ws_group if args.ws_group > 1 else "mixed-precision solves at tol 1e-6")
                                       + ("; online: a ring buffer of %d pairs on the device, training steps "
                                          "after each group" % args.ws_buffer if online else ""),
                   "net": "6 x conv3x3, 64 channels, 404 outputs", "eval_instances": args.ws_eval, "tol": args.tol},
        "zero_start_ms": zero_ms, "speedup_vs_zero_start": zero_ms / warm_ms,
        "iterations_zero": float(np.mean(zero_it)), "iterations_warm": float(np.mean(warm_it)),
        "max_rel_diff_vs_zero_fp64": max(errs), "guess_ms": guess_ms,
        "guess_rel_err_heldout": float(np.mean(guess_errs)),
        "mixed": {"zero_start_ms": 1e3 * float(np.mean(secs["zero_mixed"])),
                  "warm_start_ms": 1e3 * float(np.mean(secs["warm_mixed"])),
                  "iterations_zero": float(np.mean(its["zero_mixed"])),
                  "iterations_warm": float(np.mean(its["warm_mixed"])),
                  "speedup_warm_mixed_vs_zero_fp64": zero_ms / (1e3 * float(np.mean(secs["warm_mixed"])))},
        "training": {"generate_s": gen_s, "train_s": train_s, "first_loss": float(np.mean(losses[:10])),
                     "last_loss": float(np.mean(losses[-50:])), "conv_tflops_fp32": train_tflops,
                     "solver_iterations_per_pair": float(np.mean(ws.iterations))},
    }
    ws.close()
    print(json.dumps(line), flush=True)


def run_multirhs(args, dist):
    """Many initial states per instance: 32 right-hand sides of each of
    `args.multirhs` uneven instances solved by lq2d_solve_multi_device
    (tensor-core preconditioner), against single-right-hand-side solves of
    the same initial states (FP64 and precision mode 2) on the first
    instances."""
    import torch

    from paper_2304_04980_gb300 import lq2d

    lq2d.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    grids = synth.batch_grids(args.multirhs)

    def x0_of(idx, g):
        rng = np.random.default_rng(20000 + idx)
        return torch.from_numpy(rng.standard_normal((32, g.nodes, g.n))).to(dev)

    # The instances are processed in waves of `wave`: all 512 with their
    # 32-right-hand-side buffers would exceed the device memory.  Each wave's
    # handles are built and warmed (first solve builds the graph) untimed;
    # then each instance's solve is timed with events on the stream.
    wave = 32
    its, worst, multi_ms, launches = 0, 0.0, 0.0, 0
    probs_first, x0s_first = [], []
    for w0 in range(0, len(grids), wave):
        wprobs = [lq2d.Problem.from_grid(g) for g in grids[w0:w0 + wave]]
        wx0 = [x0_of(w0 + k, g) for k, g in enumerate(grids[w0:w0 + wave])]
        for p, x in zip(wprobs, wx0):
            p.solve_multi_device(32, x, args.tol, 2, 2, 100000, stream=stream)
        torch.cuda.synchronize()
        launches0 = sum(p.stats()["launches_total"] for p in wprobs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for p, x in zip(wprobs, wx0):
                out = p.solve_multi_device(32, x, args.tol, 2, 2, 100000, stream=stream)
                its += sum(out["iterations"])
                worst = max(worst, max(out["rel_residuals"]))
        e1.record(stream)
        torch.cuda.synchronize()
        multi_ms += e0.elapsed_time(e1) / args.steps
        launches += sum(p.stats()["launches_total"] for p in wprobs) - launches0
        if w0 == 0:
            probs_first, x0s_first = wprobs[:2], wx0[:2]
            for p in wprobs[2:]:
                p.close()
        else:
            for p in wprobs:
                p.close()
        torch.cuda.empty_cache()
    probs, x0s = probs_first, x0s_first
    # single-right-hand-side solves of the same initial states (solve time
    # only; the data update that sets each x0 is not timed)
    sub = min(2, len(grids))
    single = {}
    for mode in (0, 2):
        tot_ms, tot_its = 0.0, 0
        for idx in range(sub):
            g = grids[idx]
            sp = lq2d.Problem.from_grid(g)
            sp.set_precision(mode)
            sp.solve_device(args.tol, 2, 2, 100000, stream=stream)
            for r in range(32):
                arrays = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in g.with_x0(
                    x0s[idx][r].cpu().numpy()).arrays()]
                sp.update_device(*arrays, stream=stream)
                torch.cuda.synchronize()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                o = sp.solve_device(args.tol, 2, 2, 100000, stream=stream)
                a1.record(stream)
                torch.cuda.synchronize()
                tot_ms += a0.elapsed_time(a1)
                tot_its += o["iterations"]
            sp.close()
        single[mode] = (tot_ms, tot_its)
    # the same instances' share of the multi-right-hand-side time
    sub_ms = 0.0
    for idx in range(sub):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        probs[idx].solve_multi_device(32, x0s[idx], args.tol, 2, 2, 100000, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        sub_ms += a0.elapsed_time(a1)
    rhs = 32 * len(grids)
    line = {
        "metric": "multi-right-hand-side time-to-solve at 1e-8 rel residual (right-hand sides/s)",
        "value": rhs / (multi_ms / 1e3), "unit": "rhs/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": multi_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 iterates, f32 products, tf32 preconditioner", "data": "synthetic",
        "config": {"workload": "multirhs%d: batch family (K, N in 8..64, T in 50..200, n = 4, m = 2), 32 x0 "
                               "~ N(0, 1) per instance" % len(grids), "tol": args.tol, "S": 2, "L": 2,
                   "waves": "%d instances per wave, solve time only" % wave},
        "pcg_steps_per_rhs": its / (args.steps * rhs), "max_rel_residual": worst,
        "single_rhs_first_instances": {
            "instances": sub, "multi_ms": sub_ms,
            "fp64_ms": single[0][0], "fp64_steps_per_rhs": single[0][1] / (32 * sub),
            "mixed2_ms": single[2][0], "mixed2_steps_per_rhs": single[2][1] / (32 * sub),
            "speedup_vs_fp64": single[0][0] / sub_ms, "speedup_vs_mixed2": single[2][0] / sub_ms},
        "gpu_launches": launches,
    }
    for p in probs:
        p.close()
    print(json.dumps(line), flush=True)


def run_mrhs_apply(args):
    """D_S r of 32 right-hand sides at once (lq2d_apply_precond_multi_device),
    `args.mrhs_apply` times after one untimed application."""
    import torch

    from paper_2304_04980_gb300 import lq2d

    lq2d.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = synth.workload(args.workload)
    prob = lq2d.Problem.from_grid(g)
    r = torch.from_numpy(synth.random_vector((32, g.T + 1, g.nodes, g.n), seed=7)).to(dev)
    q = torch.empty_like(r)
    prob.apply_precond_multi_device(32, 2, 2, r, q, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.mrhs_apply):
        prob.apply_precond_multi_device(32, 2, 2, r, q, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.mrhs_apply, 1)
    print(json.dumps({"metric": "32-right-hand-side D_S r (ms per application)", "value": ms, "unit": "ms",
                      "config": {"workload": args.workload, "rhs": 32, "S": 2, "L": 2},
                      "applications": args.mrhs_apply}), flush=True)
    prob.close()


def main():
    args = parse_args()
    if args.mrhs_apply > 0:
        run_mrhs_apply(args)
        return
    if args.warmstart > 0:
        run_warmstart(args, Dist())
        return
    if args.batch > 0:
        run_batch(args, Dist())
        return
    if args.multirhs > 0:
        run_multirhs(args, Dist())
        return
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)   # rank 0 only; no process group needed
        return
    import torch
    if dist.world > 1:
        torch.cuda.set_device(dist.local)
    dist.init("nccl")
    try:
        run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
