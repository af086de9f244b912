"""Benchmark: one step = one pass of black-box HBS compression (Algorithm 2) on one matrix.

Workload (default): dense 2D log kernel A_ij = log|x_i - x_j| (A_ii = 0) on N = 32768 points
evenly spaced in angle on r(theta) = 1 + 0.3 cos 5 theta, rank parameter r = 40, s = 120 test
vectors, leaf size 64 (the largest power-of-two split with leaf <= s - r), all in FP64.
A step draws Omega and Psi (Philox, 2 launches), forms Y = A Omega and Z = A^* Psi (2 FP64
GEMM launches) and runs the sweep (two launches per tree level, 10 levels). A (8.6 GB) is
resident in HBM before timing and is streamed in full every step, so no L2 flush is needed.
The same run also times the mixed precisions on the same matrix stored in FP32 (``modes``):
"mixed" (bf16x6 tensor-core products, FP32 node arithmetic around the FP64 nullspace and
pseudo-inverse) and "tc64" (bf16x6 products, FP64 sweep), each with its accuracy against A
and against the FP64 result. ``--only MODE`` times one mode (used for profiling).

Metric: compress throughput N*s / T (sample rows x columns consumed per second) with the
compress time T in ms_per_step. ``e2e`` repeats the step through the same C ABI calls with A in
pinned host memory, copying A in and the factors out inside the timed region. ``cpu_baseline``
and ``--impl reference`` time the FP64 oracle on the host cores on a bounded sample of the same
workload (stated in the ``sample`` field) and scale it to the full workload.

Multi-GPU (torchrun): each rank compresses its own replica; ranks never exchange data.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HBS compress time (ms) & N·s/sec at stated rel. error, mixed/batched vs FP64"
UNIT = "N*s/s"
N_DEF, R_DEF, S_DEF, LEAF_DEF, SEED = 32768, 40, 120, 64, 220502990 + 200
SM_COUNT_GB300 = 152
FP64_DFMA_PER_CLK_PER_SM = 2          # GB300: FP64 at 1/64 of the FP32 rate (1.25 TF nominal)
GEMM_READ_8192 = 549.24e6             # dram bytes read by one sample_gemm_f64 launch, N = 8192
GEMM_WRITE_8192 = 41.77e6             # dram bytes written (split-K partials) by that launch
def measured_peaks():
    """Dense bf16 (sustained) and HBM copy peaks measured on the GB300s
    (MEASURED_PEAKS.json beside this file, written by the pool's driver), else the fallback of one
    earlier GB300 measurement (1.7 PFLOP/s sustained, 6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1700.0, 6800.0, "fallback"


BF16_TFLOPS_SUSTAINED, HBM_GBS, PEAKS_SOURCE = measured_peaks()
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # derived FP64 peak: SMs x DFMA/clk x 2 flop x clock
DF32_SLOTS = 15                       # FP32 instructions of one double-float multiply-add


def tree_nodes(N, leaf):
    L = 0
    while -(-N // 2 ** L) > leaf:
        L += 1
    return L


def node_flops(n, r, s, root=False):
    """Algorithmic flops of one node of the sweep (Householder counts; the D and merge terms in
    the form the reduced-precision finish evaluates them, 12 r n^2 + 12 n r s)."""
    lq = 2 * n * n * (s - n / 3)                 # QR of Omega_tau^* (s x n)
    stream = 4 * n * n * s - 2 * n ** 3          # n rows through n reflectors
    solve = n ** 3                               # rows of Y Omega^+ against L_1
    if root:
        return lq + stream + solve
    colqr = 2 * r * r * (n - r / 3) + 4 * n * r * r - 4 * r ** 3 / 3
    dblk = 12 * r * n * n
    merge = 12 * n * r * s
    return 2 * (lq + stream + solve + colqr) + dblk + merge


def sweep_flops(N, r, s, leaf):
    L = tree_nodes(N, leaf)
    total = 0.0
    for level in range(L, -1, -1):
        cnt = 2 ** level
        if level == L and L > 0:
            big = -(-N // 2 ** L)
            small = N // 2 ** L
            n_big = N - small * cnt
            total += n_big * node_flops(big, r, s) + (cnt - n_big) * node_flops(small, r, s)
        elif level == 0:
            total += node_flops(2 * r if L > 0 else N, r, s, root=True)
        else:
            total += cnt * node_flops(2 * r, r, s)
    return total


# Per-phase flops of one node, in the form each kernel evaluates the step (Algorithm 2):
# side = LQ of one test block + its n sample rows through the reflectors + the solve with L_1;
# bases = col(., r) of one side; D and merges as the FP64 finish forms them (P, Q, R, M, D; then
# S - op(D) T and the two basis products per pass) or as the reduced finishes do (D with U^* D
# and (D V)^*, then [B^*, -H][S; T]).
def side_flops(n, s):
    return side_lq_flops(n, s) + side_rows_flops(n, s)


def side_lq_flops(n, s):
    """The LQ of one n x s test block."""
    return 2 * n * n * (s - n / 3)


def side_rows_flops(n, s):
    """Its n sample rows through the n reflectors, and the back substitution."""
    return (4 * n * n * s - 2 * n ** 3) + n ** 3


def bases_flops(n, r):
    return 2 * r * r * (n - r / 3) + 4 * n * r * r - 4 * r ** 3 / 3


def d_flops(n, r, reduced):
    return 12 * r * n * n if reduced else 6 * r * n * n + 4 * r * r * n


def merge_flops(n, r, s, reduced):
    return 12 * n * r * s if reduced else 4 * n * n * s + 8 * n * r * s


def sweep_launches(N, r, s, leaf, tuning, reduced):
    """Kernel launches of one sweep: per height the side, bases, D (two kernels in FP64) and
    merge kernels (the root height runs all of them too)."""
    return len(tuning) * ((1 + 3) if reduced else (1 + 4))


def df32_fits(n, r):
    """Whether the double-float D and merge tiles of nodes of n rows fit 227 KB of shared memory
    (the library runs the FP64 finish on heights where they do not)."""
    dchain = r * (n + 1) + r * n + 2 * n * r + n * (n + 1) + n * n
    merge = 2 * n * 32 + 3 * n * r + r * 32
    return 8 * max(dchain, merge) <= 227 * 1024


def sweep_phase_flops(N, r, s, leaf, reduced):
    """Per height (finest first): flops of the side, bases, D and merge phases. ``reduced`` is
    False (FP64 finish), "fp32" or "df32"."""
    L = tree_nodes(N, leaf)
    out = []
    for level in range(L, -1, -1):
        cnt = 2 ** level
        if level == L and L > 0:
            big, small = -(-N // cnt), N // cnt
            n_big = N - small * cnt
            groups = [(big, n_big), (small, cnt - n_big)]
        elif level == 0:
            groups = [(2 * r if L > 0 else N, 1)]
        else:
            groups = [(2 * r, cnt)]
        if level == 0:
            n = groups[0][0]
            out.append([side_flops(n, s), 0.0, 0.0, 0.0])
            continue
        ph = [0.0, 0.0, 0.0, 0.0]
        red = bool(reduced) and (reduced != "df32" or df32_fits(max(n for n, _ in groups), r))
        for n, c in groups:
            ph[0] += c * 2 * side_flops(n, s)
            ph[1] += c * 2 * bases_flops(n, r)
            ph[2] += c * d_flops(n, r, red)
            ph[3] += c * merge_flops(n, r, s, red)
        out.append(ph)
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_host_numa(gpu_id):
    """NUMA node of the GPU's PCI device and the CPUs of that node (from sysfs), if known."""
    info = {"gpu_numa_node": None, "node_cpus": None, "process_cpus": None}
    try:
        info["process_cpus"] = len(os.sched_getaffinity(0))
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu_id), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().lower()
        if bus:
            bus = bus[-12:] if len(bus) > 12 else bus          # domain:bus:dev.fn
            path = f"/sys/bus/pci/devices/{bus}/numa_node"
            if os.path.exists(path):
                node = int(open(path).read().strip())
                info["gpu_numa_node"] = node
                if node >= 0:
                    cl = open(f"/sys/devices/system/node/node{node}/cpulist").read().strip()
                    cpus = set()
                    for part in cl.split(","):
                        a, _, b = part.partition("-")
                        cpus.update(range(int(a), int(b or a) + 1))
                    info["node_cpus"] = sorted(cpus)
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return info


class numa_local:
    """Runs the block on the CPUs of the GPU's NUMA node (so that pages pinned there are local to
    the GPU), then restores the affinity."""

    def __init__(self, info):
        self.cpus = info.get("node_cpus")
        self.saved = None

    def __enter__(self):
        if self.cpus:
            try:
                self.saved = os.sched_getaffinity(0)
                allowed = set(self.cpus) & self.saved
                if allowed:
                    os.sched_setaffinity(0, allowed)
            except OSError:
                self.saved = None
        return self

    def __exit__(self, *exc):
        if self.saved:
            os.sched_setaffinity(0, self.saved)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload (cpu_baseline and --impl reference)

def oracle_sample_time(N, r, s, leaf, rows=4096, sweep_N=8192, workload="logkernel", measured=None):
    """Seconds the FP64 oracle would take for the full workload, from a bounded sample:
    Philox rows and sampling products for ``rows`` of the N rows, and the sweep of a
    ``sweep_N``-point problem of the same r, s, leaf, each scaled by its share of the work.
    With ``measured`` (a list), the sample's own seconds are appended to it."""
    import numpy as np
    from hbs_inputs import double_layer_rows, gaussian, log_kernel_rows
    from oracle import philox
    from oracle.compress import compress
    from oracle.sample import sample_dense

    idx = np.arange(rows)
    A_rows = (double_layer_rows if workload == "doublelayer" else log_kernel_rows)(N, idx)
    t0 = time.perf_counter()
    Om_rows = philox.gaussian_matrix(N, s, 0, SEED, rows=idx)
    Ps_rows = philox.gaussian_matrix(N, s, 1, SEED, rows=idx)
    m_rng = time.perf_counter() - t0
    Om = np.tile(Om_rows, (N // rows + 1, 1))[:N]           # full-height Omega stand-in
    t0 = time.perf_counter()
    sample_dense(A_rows, Om, Ps_rows)                        # rows x N block of both products
    m_smp = time.perf_counter() - t0
    x = [gaussian((sweep_N, s), 17 + i) for i in range(4)]
    t0 = time.perf_counter()
    compress(*x, r, leaf)
    m_sw = time.perf_counter() - t0
    if measured is not None:
        measured.append(m_rng + m_smp + m_sw)
    t_rng, t_smp = m_rng * N / rows, m_smp * N / rows
    t_sw = m_sw * sweep_flops(N, r, s, leaf) / sweep_flops(sweep_N, r, s, leaf)
    sample = (f"Philox draws and both sampling products for {rows} of {N} rows, sweep of a "
              f"{sweep_N}-point problem (r={r}, s={s}, leaf {leaf}); scaled to N={N} by rows and "
              f"by sweep flops")
    return t_rng + t_smp + t_sw, sample


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args, N, r, s, leaf):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_time(N, r, s, leaf)
    times, measured, sample = [], [], ""
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        t, sample = oracle_sample_time(N, r, s, leaf, measured=measured)
        times.append(t)
    wall = time.perf_counter() - wall0
    t = statistics.mean(times)
    value = N * s / t
    # a step is one bounded sample of the workload: its time is what the step took, and its work
    # is the fraction of a full step that the sample represents (value x time = work done)
    step_s = statistics.mean(measured)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "work_fraction_per_step": step_s / t, "ms_per_full_step_scaled": t * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"log-kernel N={N} r={r} s={s} leaf={leaf} FP64 dense",
                       "N": N, "r": r, "s": s, "leaf": leaf, "precision": "fp64",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample, "wall_s": wall},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------

MODES = {
    "fp64": dict(sample=0, sweep=0, a="f64",
                 what="FP64 products on the FP64 pipe + FP64 sweep"),
    "mixed": dict(sample=2, sweep=2, a="f32",
                  what="A stored FP32; bf16x6 products on tcgen05 tensor cores; sweep with FP64 "
                       "nullspace LQ / pseudo-inverse (sample rows through it in double-float) and "
                       "FP32 bases, D_tau and merges"),
    "tc64": dict(sample=2, sweep=0, a="f32",
                 what="A stored FP32; bf16x6 products on tcgen05 tensor cores; FP64 sweep"),
    "oz64": dict(sample=3, sweep=3, a="f64",
                 what="A stored FP64; FP64-class products from 7 exact 8-bit digits per entry "
                      "(28 FP16 digit-pair products on tcgen05 tensor cores, exact FP32 sums); "
                      "FP64 sweep"),
    "cmp": dict(sample=4, sweep=4, a="f64",
                what="A stored FP64; products from 5 exact 8-bit digits per entry, one exponent "
                     "per 64 x 64 block of A (15 FP16 digit-pair products on tcgen05 tensor cores, "
                     "exact FP32 sums); sweep with "
                     "FP64 nullspace LQ / pseudo-inverse and bases, double-float (compensated "
                     "FP32) sample rows through the LQ, D_tau and merges"),
    "mixed3": dict(sample=1, sweep=1, a="f32",
                   what="A stored FP32; bf16x3 products on tcgen05 tensor cores; sweep with FP64 "
                        "nullspace LQ / pseudo-inverse (sample rows through it in double-float) "
                        "and FP32 bases, D_tau and merges"),
}
FINISH = {0: "fp64", 1: "fp32", 2: "fp32", 3: "fp64", 4: "df32"}


def peaks_now(hb):
    """Pipe peaks: derived from the unit counts and the 2070 MHz maximum clock, and measured now
    by the library's FMA-chain probe (hbs_probe_peaks)."""
    fp64_probe, fp32_probe = hb.hbs_probe_peaks()
    fp32 = SM_COUNT_GB300 * 128 * 2 * 2070e6 / 1e12
    return {"fp64_derived": FP64_TFLOPS, "fp32_derived": fp32,
            "df32_derived": fp32 / DF32_SLOTS, "fp64_probe": fp64_probe, "fp32_probe": fp32_probe,
            "df32_from_probe": fp32_probe / DF32_SLOTS, "fp64_dmma_probe": hb.hbs_probe_dmma(),
            # cycles per M = N = 128, K = 16 tcgen05 MMA issued by one thread, alone and beside
            # FP32 work (the bound of the drain-heavy digit GEMM)
            "mma_issue_cycles": hb.hbs_probe_mma_issue()}


def side_split_per_height(N, r, s, leaf):
    """Per height (finest first): (LQ flops, sample-row flops, largest node) of the side phase."""
    L = tree_nodes(N, leaf)
    out = []
    for level in range(L, -1, -1):
        cnt = 2 ** level
        if level == L and L > 0:
            big, small = -(-N // cnt), N // cnt
            groups = [(big, N - small * cnt), (small, cnt - (N - small * cnt))]
        elif level == 0:
            groups = [(2 * r if L > 0 else N, 1)]
        else:
            groups = [(2 * r, cnt)]
        sides = 1 if level == 0 else 2
        out.append((sum(c * sides * side_lq_flops(n, s) for n, c in groups),
                    sum(c * sides * side_rows_flops(n, s) for n, c in groups),
                    max(n for n, _ in groups)))
    return out


def sweep_roofline(phase_ms, N, r, s, leaf, finish, peaks, tuning=None):
    """Roofline of the sweep's four phases from a hbs_profile_sweep run: algorithmic flops
    (sweep_phase_flops) per height and phase over the CUDA-event time, against the derived peak
    of the pipe each phase runs on (FP64; FP32 for the plain mixed finish; double-float: the FP32
    peak over the 15 FP32 instructions of one double-float multiply-add). With a reduced finish
    the side phase runs its LQ in FP64 and, at heights of the one-CTA form (tuning R > 0), its
    sample rows in double-float: its fraction is then the time those flops need at their pipes'
    peaks over the measured time."""
    flops = sweep_phase_flops(N, r, s, leaf, False if finish == "fp64" else finish)
    names = ("side", "bases", "D", "merge")
    pipe = {"side": "fp64", "bases": "fp32" if finish == "fp32" else "fp64",
            "D": finish, "merge": finish}
    peak = {p: peaks[p + "_derived"] for p in ("fp64", "fp32", "df32")}
    # the side phase's ideal time per height (s), by pipe
    split = side_split_per_height(N, r, s, leaf)
    side_ideal = []
    for h, (lq, rows, nmax) in enumerate(split):
        df_rows = (finish != "fp64" and tuning is not None and h < len(tuning) and tuning[h] > 0
                   and (finish == "fp32" or df32_fits(nmax, r)))
        side_ideal.append(lq / (peak["fp64"] * 1e12)
                          + rows / ((peak["df32"] if df_rows else peak["fp64"]) * 1e12))
    if finish != "fp64":
        pipe["side"] = "fp64 LQ + df32 sample rows (one-CTA heights)"
    per_kernel = {}
    for k, nm in enumerate(names):
        ms = sum(h[k] for h in phase_ms)
        fl = sum(f[k] for f in flops)
        ach = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        if nm == "side" and finish != "fp64":
            frac = sum(side_ideal) / (ms * 1e-3) if ms > 0 else 0.0
            fbh = [round(t / (h[0] * 1e-3), 3) if h[0] > 0 else None
                   for h, t in zip(phase_ms, side_ideal)]
            pk = None
        else:
            frac = ach / peak[pipe[nm]]
            fbh = [round((f[k] / (h[k] * 1e-3) / 1e12) / peak[pipe[nm]], 3)
                   if h[k] > 0 and f[k] > 0 else None for h, f in zip(phase_ms, flops)]
            pk = peak[pipe[nm]]
        per_kernel[nm] = {"ms": ms, "gflop": fl / 1e9, "achieved_tflops": ach,
                          "pipe": pipe[nm], "peak_tflops": pk, "frac": frac,
                          "frac_by_height": fbh,
                          "ms_by_height": [round(h[k], 4) for h in phase_ms]}
    tot_ms = sum(sum(h) for h in phase_ms)
    tot_fl = sum(sum(f) for f in flops)
    return {"finish": finish, "per_kernel": per_kernel,
            "total": {"ms": tot_ms, "gflop": tot_fl / 1e9,
                      "achieved_tflops": tot_fl / (tot_ms * 1e-3) / 1e12,
                      "frac_of_fp64_peak": tot_fl / (tot_ms * 1e-3) / 1e12 / peak["fp64"]},
            "peak_source": "derived: 152 SMs x (2 DFMA | 128 FFMA)/clk x 2 flop x 2070 MHz; "
                           "double-float = FP32 / 15 instructions per multiply-add",
            "timing": "CUDA events between the launches of one extra sweep with plain launches "
                      "(hbs_profile_sweep)"}


def run_batched(hb, torch, items=256, seed=SEED + 400, reps=3):
    """256 independent exact-HBS operators (N in {2048, 4096, 8192, 16384}, block rank k in
    [8, 32]) compressed with r = k + 5 (Section 4: r = k + p, p = 5 usually suffices; with p = 0
    the method amplifies rounding ~1e7-fold), s = 3r, leaf = largest power of two <= 2r, applied
    as black boxes (their telescoping factors loaded into a handle, applied by Algorithm 1),
    sampled by one batched apply per direction, then compressed as one batch: the side, bases,
    D and merge launches of each tree height cover all 256 trees, replayed from a CUDA graph,
    side shapes autotuned. Returns timings of the sweep alone (T2) and of drawing + black-box
    sampling + sweep (T1), FP64 and mixed."""
    import numpy as np
    from hbs_inputs import exact_hbs_packed_torch
    rng = np.random.default_rng(seed)
    Ns = rng.choice([2048, 4096, 8192, 16384], size=items)
    ks = rng.integers(8, 33, size=items)
    probs, gprobs, Oms, Pss, Ys, Zs, packed = [], [], [], [], [], [], []
    for i in range(items):
        N, k = int(Ns[i]), int(ks[i])
        r = k + 5
        leaf = 1 << int(np.floor(np.log2(2 * r)))
        s = 3 * r
        bufs = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
        Oms.append(bufs[0]), Pss.append(bufs[1]), Ys.append(bufs[2]), Zs.append(bufs[3])
        probs.append(hb.Problem(N, r, s, leaf, *bufs))
        gprobs.append(hb.Problem(N, k, s, leaf, *bufs))
        packed.append(exact_hbs_packed_torch(N, leaf, k, seed + i, "cuda"))
    gen = hb.hbs_plan(gprobs)                          # the black boxes: generator factors
    hb.hbs_load_factors(gen, torch.cat(packed))
    del packed
    total_ns = float(sum(int(p.N) * int(p.s) for p in probs))

    def draw_and_sample():
        for i, p in enumerate(probs):
            hb.hbs_draw_gaussian(p.N, p.s, 0, seed + 7 * i, Oms[i])
            hb.hbs_draw_gaussian(p.N, p.s, 1, seed + 7 * i, Pss[i])
        hb.hbs_apply_batch(gen, Oms, Ys)
        hb.hbs_apply_batch(gen, Pss, Zs, trans=True)

    draw_and_sample()
    out = {"items": items, "total_N_s": total_ns,
           "shapes": "N in {2048,4096,8192,16384}, k in [8,32], r=k+5, s=3r, leaf=pow2<=2r",
           "heights": None}
    for name, prec in (("fp64", 0), ("compensated", 4), ("mixed", 2)):
        h = hb.hbs_plan(probs, precision=prec)
        hb.hbs_execute(h, probs)
        hb.hbs_autotune(h)
        hb.hbs_execute(h, probs)                       # graph captured with the tuned slicing
        hb.hbs_sync_status(h)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        for _ in range(reps):
            hb.hbs_execute(h, probs)
        e[1].record()
        e[2].record()
        for _ in range(reps):
            draw_and_sample()
            hb.hbs_execute(h, probs)
        e[3].record()
        torch.cuda.synchronize()
        hb.hbs_sync_status(h)
        t2 = e[0].elapsed_time(e[1]) / reps
        t1 = e[2].elapsed_time(e[3]) / reps
        # accuracy: one probe column per operator, ||(A~ - A) x|| / ||A x|| with A the black box
        xs = [torch.randn((p.N, 1), dtype=torch.float64, device="cuda") for p in probs]
        ya = [torch.empty_like(x) for x in xs]
        yb = [torch.empty_like(x) for x in xs]
        hb.hbs_apply_batch(gen, xs, ya)
        hb.hbs_apply_batch(h, xs, yb)
        errs = [float(torch.linalg.norm(b - a) / torch.linalg.norm(a)) for a, b in zip(ya, yb)]
        out["heights"] = len(hb.hbs_get_tuning(h))
        out[name] = {"T2_sweep_ms": t2, "T1_total_ms": t1, "value_T2": total_ns / (t2 / 1e3),
                     "value_T1": total_ns / (t1 / 1e3), "rel_error_probe_max": max(errs),
                     "rel_error_probe_median": float(np.median(errs)),
                     "tuned_row_slices": hb.hbs_get_tuning(h),
                     # every tree of the batch in each launch; the sweep replayed from one graph
                     "launches_per_height": "side 1, bases 1, D " + ("2 (FP64)" if name == "fp64" else "1")
                                            + ", merges 1"}
        h.free()
    gen.free()
    return out


def run_config3(hb, torch, steps, warmup, N=65536, r=R_DEF, s=S_DEF, leaf=LEAF_DEF,
                seed=SEED + 300):
    """The mixed-precision workload at N = 65536 (log kernel, r = 40, s = 120, leaf 64): "mixed"
    (A stored FP32, 17.2 GB; bf16x6 products; FP32 bases, D_tau, merges around the FP64 LQ),
    "mixed3" (the same with bf16x3 products, the split the workload names) and "cmp" (A stored
    FP64; 5-digit products; double-float D_tau and merges), each timed per step (draws, products,
    sweep) and held against the dense A and against the FP64 result (FP64-pipe products and FP64
    sweep, run once) by 20 power steps (Section 5). Device-timed, A resident and streamed every
    step (larger than L2)."""
    from hbs_inputs import log_kernel_torch
    A = log_kernel_torch(N, "cuda")
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    prob = hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)
    out = {"N": N, "r": r, "s": s, "leaf": leaf, "A_fp64_gb": A.numel() * 8 / 1e9,
           "A_fp32_gb": A.numel() * 4 / 1e9}

    def draw():
        hb.hbs_draw_gaussian(N, s, 0, seed, Om)
        hb.hbs_draw_gaussian(N, s, 1, seed, Ps)

    def power_norm(apply_B, apply_Bt, nsteps=20):
        g = torch.Generator(device="cuda").manual_seed(3)
        v = torch.randn((N, 1), dtype=torch.float64, device="cuda", generator=g)
        for _ in range(nsteps):
            v = apply_Bt(apply_B(v / torch.linalg.norm(v)))
        return float(torch.sqrt(torch.linalg.norm(v)))

    def apply_h(h, x, trans=False):
        o = torch.empty_like(x)
        hb.hbs_apply(h, x, o, trans=trans)
        return o

    draw()
    hb.hbs_sample_products(A, s, Om, Ps, Y, Z, precision=0)
    h64 = hb.hbs_compress([prob], precision=0)
    hb.hbs_sync_status(h64)
    nA = power_norm(lambda x: A @ x, lambda x: A.T @ x)
    n64 = power_norm(lambda x: apply_h(h64, x), lambda x: apply_h(h64, x, True))
    out["fp64_once"] = {"rel_error": power_norm(lambda x: apply_h(h64, x) - A @ x,
                                                lambda x: apply_h(h64, x, True) - A.T @ x) / nA}
    A32 = None
    for mode in ("mixed", "mixed3", "cmp"):
        cfg = MODES[mode]
        if cfg["a"] == "f32" and A32 is None:
            A32 = A.float()
        Aop = A if cfg["a"] == "f64" else A32
        h = hb.hbs_plan([prob], precision=cfg["sweep"])
        draw()
        hb.hbs_sample_products(Aop, s, Om, Ps, Y, Z, precision=cfg["sample"])
        hb.hbs_execute(h, [prob])
        hb.hbs_autotune(h)

        def step():
            draw()
            hb.hbs_sample_products(Aop, s, Om, Ps, Y, Z, precision=cfg["sample"])
            hb.hbs_execute(h, [prob])

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        hb.hbs_sync_status(h)
        hb.hbs_sample_sync()
        ms = e0.elapsed_time(e1) / steps
        out[mode] = {"ms_per_step": ms, "value": N * s / (ms / 1e3), "steps": steps,
                     "rel_error": power_norm(lambda x: apply_h(h, x) - A @ x,
                                             lambda x: apply_h(h, x, True) - A.T @ x) / nA,
                     "vs_fp64": power_norm(lambda x: apply_h(h, x) - apply_h(h64, x),
                                           lambda x: apply_h(h, x, True) - apply_h(h64, x, True)) / n64,
                     "what": cfg["what"]}
        h.free()
    h64.free()
    del A, A32, Om, Ps, Y, Z
    torch.cuda.empty_cache()
    return out


def run_apply(hb, torch, logN=22, k=45, leaf=64, seed=SEED + 600, reps=5):
    """Algorithm 1 on its own: Out = A~ X and A~^* X for an exact-HBS operator in telescoping
    form (N = 2^22, rank 45, leaf 64; the factors loaded into a handle) and X with 1, 16 and 150
    columns. Bytes: every factor read once, X read once, Out written once (the r-row workspace of
    the two passes is left out: 2 (2^(L+1) - 2) r c doubles, under 1 % of the factors at c = 1).
    Flops: 2 c per factor entry. Device-timed (CUDA events), inputs resident."""
    from hbs_inputs import exact_hbs_packed_torch
    N = 1 << logN
    bufs = [torch.empty((N, 3 * k), dtype=torch.float64, device="cuda") for _ in range(4)]
    gen = hb.hbs_plan([hb.Problem(N, k, 3 * k, leaf, *bufs)])   # the samples are not used
    del bufs
    hb.hbs_load_factors(gen, exact_hbs_packed_torch(N, leaf, k, seed, "cuda"))
    fbytes = hb.hbs_factor_bytes(gen)
    rows = []
    for c in (1, 16, 150):
        X = torch.randn((N, c), dtype=torch.float64, device="cuda")
        Out = torch.empty_like(X)
        row = {"ncols": c}
        for trans in (False, True):
            hb.hbs_apply(gen, X, Out, trans=trans)        # warm-up (and workspace growth)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                hb.hbs_apply(gen, X, Out, trans=trans)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            nbytes = fbytes + 2 * N * c * 8
            flops = 2.0 * c * fbytes / 8
            row["trans" if trans else "plain"] = {
                "ms": ms, "GB_per_s": nbytes / ms / 1e6, "hbm_frac": nbytes / ms / 1e6 / HBM_GBS,
                "GFLOP_per_s": flops / ms / 1e6, "fp64_frac": flops / ms / 1e9 / FP64_TFLOPS}
        rows.append(row)
        del X, Out
    gen.free()
    return {"N": N, "factor_bytes": fbytes, "rows": rows}


def run_scaling(hb, torch, logN_list, k=45, r=50, s=150, leaf=64, seed=SEED + 500, reps=2):
    """Linear-complexity check (Section 4.4, Section 5 summary): an exact-HBS operator of block
    rank k = 45 (N = 2^16 .. 2^22, leaf 64) applied as a black box by Algorithm 1 on its loaded
    telescoping factors, never formed densely; compressed with r = 50 = k + 5, s = 150 in FP64
    and in the mixed precision. Per N: sweep time (T2), draw + black-box sampling + sweep (T1),
    and the accuracy against the operator on 4 random probe columns."""
    from hbs_inputs import exact_hbs_packed_torch
    rows = []
    for logN in logN_list:
        N = 1 << logN
        bufs = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
        Om, Ps, Y, Z = bufs
        prob = hb.Problem(N, r, s, leaf, *bufs)
        gen = hb.hbs_plan([hb.Problem(N, k, s, leaf, *bufs)])
        hb.hbs_load_factors(gen, exact_hbs_packed_torch(N, leaf, k, seed + logN, "cuda"))

        def draw_and_sample():
            hb.hbs_draw_gaussian(N, s, 0, seed, Om)
            hb.hbs_draw_gaussian(N, s, 1, seed, Ps)
            hb.hbs_apply(gen, Om, Y)
            hb.hbs_apply(gen, Ps, Z, trans=True)

        draw_and_sample()
        row = {"N": N}
        for name, prec in (("fp64", 0), ("compensated", 4), ("mixed", 2)):
            h = hb.hbs_plan([prob], precision=prec)
            hb.hbs_execute(h, [prob])
            hb.hbs_sync_status(h)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            e[0].record()
            for _ in range(reps):
                hb.hbs_execute(h, [prob])
            e[1].record()
            e[2].record()
            for _ in range(reps):
                draw_and_sample()
                hb.hbs_execute(h, [prob])
            e[3].record()
            torch.cuda.synchronize()
            hb.hbs_sync_status(h)
            x = torch.randn((N, 4), dtype=torch.float64, device="cuda")
            ya, yb = torch.empty_like(x), torch.empty_like(x)
            hb.hbs_apply(gen, x, ya)
            hb.hbs_apply(h, x, yb)
            t2 = e[0].elapsed_time(e[1]) / reps
            t1 = e[2].elapsed_time(e[3]) / reps
            row[name] = {"T2_sweep_ms": t2, "T1_total_ms": t1, "ns_per_index_T2": t2 * 1e6 / N,
                         "rel_error_probe": float(torch.linalg.norm(yb - ya) / torch.linalg.norm(ya))}
            h.free()
        gen.free()
        del bufs, Om, Ps, Y, Z
        torch.cuda.empty_cache()
        rows.append(row)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hbs", choices=["hbs", "reference"])
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--only", default=None,
                    help="comma-separated precision modes to time (of " + ", ".join(sorted(MODES))
                         + "); default: fp64 headline plus the others")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the N = 65536 mixed-precision workload")
    ap.add_argument("--no-apply", action="store_true",
                    help="skip Algorithm 1 on the N = 2^22 exact-HBS operator")
    ap.add_argument("--workload", default="logkernel",
                    choices=["logkernel", "doublelayer", "scaling", "batched", "apply"],
                    help="logkernel: the timed N = 32768 log-kernel step (default); doublelayer: "
                         "the Section 5.1 boundary-integral operator with r = 30, m = 60, s = 90; "
                         "scaling: black-box exact-HBS compression for N = 2^16 .. 2^22; "
                         "batched: the 256-operator batch alone; apply: Algorithm 1 on an "
                         "N = 2^22 exact-HBS operator with 1, 16 and 150 columns")
    ap.add_argument("--max-logN", type=int, default=22,
                    help="largest log2 N of the scaling workload; the N of the apply workload")
    args = ap.parse_args()
    only = [m.strip() for m in args.only.split(",")] if args.only else None
    if only and any(m not in MODES for m in only):
        ap.error("--only takes modes from " + ", ".join(sorted(MODES)))
    N, r, s, leaf = args.N, R_DEF, S_DEF, LEAF_DEF
    if args.workload == "doublelayer":
        r, s, leaf = 30, 90, 60
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, N, r, s, leaf)
        return

    import torch
    import torch.distributed as dist

    import paper_2205_02990_gb300 as hb
    from hbs_inputs import double_layer_torch, log_kernel_torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hb.load()
    if args.workload == "apply":
        out = run_apply(hb, torch, logN=args.max_logN)
        if rank == 0:
            print(json.dumps({"workload": "Algorithm 1, exact-HBS operator, rank 45, leaf 64",
                              "apply": out}), flush=True)
        return
    if args.workload == "batched":
        out = run_batched(hb, torch)
        if rank == 0:
            print(json.dumps({"workload": "256 exact-HBS operators, batched", "batched": out}),
                  flush=True)
        return
    if args.workload == "scaling":
        rows = run_scaling(hb, torch, list(range(16, args.max_logN + 1)))
        if rank == 0:
            print(json.dumps({"workload": "exact-HBS black box, k=45, r=50, s=150, leaf 64",
                              "unit": "ms", "rows": rows}), flush=True)
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.current_stream()
    modes = only or ["fp64", "oz64", "cmp", "mixed", "tc64"]
    peaks = peaks_now(hb)
    A = (double_layer_torch if args.workload == "doublelayer" else log_kernel_torch)(N, "cuda")
    A32 = A.float() if any(MODES[m]["a"] == "f32" for m in modes) else None
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    L = tree_nodes(N, leaf)
    seed = SEED + 1000 * rank
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_id = visible[local].strip() if local < len(visible) and visible[local].strip() else local

    def timed(mode, steps, warmup, sample_clocks):
        cfg = MODES[mode]
        Aop = A if cfg["a"] == "f64" else A32
        prob = hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)
        h = hb.hbs_plan([prob], precision=cfg["sweep"])
        hb.hbs_draw_gaussian(N, s, 0, seed, Om)            # inputs for the one-time tuning
        hb.hbs_draw_gaussian(N, s, 1, seed, Ps)
        hb.hbs_sample_products(Aop, s, Om, Ps, Y, Z, precision=cfg["sample"])
        hb.hbs_execute(h, [prob])
        hb.hbs_autotune(h)                                 # side shape per height (plan time)
        plain_steps = min(steps, 5)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(plain_steps)]

        def step(A_src=None):
            # the library's one call: draws, products, sweep, with the leaves' test-block LQ on
            # a second stream while the products run
            hb.hbs_sample_execute(h, Aop if A_src is None else A_src, seed,
                                  precision=cfg["sample"], problems=[prob])

        def plain_step(i=None, A_src=None):
            # the same work as separate calls, nothing overlapped; the products between events
            hb.hbs_draw_gaussian(N, s, 0, seed, Om)
            hb.hbs_draw_gaussian(N, s, 1, seed, Ps)
            if i is not None:
                ev[i][0].record(stream)
            hb.hbs_sample_products(Aop if A_src is None else A_src, s, Om, Ps, Y, Z,
                                   precision=cfg["sample"])
            if i is not None:
                ev[i][1].record(stream)
            hb.hbs_execute(h, [prob])

        def run_timed(fn, k):
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(k):
                fn(i)
            b.record(stream)
            barrier()
            return max_over_ranks(a.elapsed_time(b) / 1e3)

        for _ in range(warmup):
            step()
        hb.hbs_sync_status(h)
        hb.hbs_sample_sync()
        clk = ClockSampler(gpu_id) if sample_clocks else None
        if clk:
            clk.__enter__()
        elapsed = run_timed(lambda i: step(), steps)
        if clk:
            clk.__exit__(None, None, None)
        plain_step()
        elapsed_plain = run_timed(plain_step, plain_steps)
        hb.hbs_sync_status(h)
        hb.hbs_sample_sync()
        per_launch = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / (2 * plain_steps)
        phases = hb.hbs_profile_sweep(h)                   # one more sweep, events per launch

        def products_ms():                                 # of the steps timed with events
            return sum(a.elapsed_time(b) for a, b in ev) / plain_steps

        return dict(h=h, step=step, plain_step=plain_step, plain_steps=plain_steps,
                    elapsed=elapsed, elapsed_plain=elapsed_plain, per_launch=per_launch,
                    products_ms=products_ms, clocks=clk.summary() if clk else None,
                    tuning=hb.hbs_get_tuning(h),
                    sweep=sweep_roofline(phases, N, r, s, leaf, FINISH[cfg["sweep"]], peaks,
                                         hb.hbs_get_tuning(h)))

    def power_norm(apply_B, apply_Bt, steps=20):
        g = torch.Generator(device="cuda").manual_seed(3)
        v = torch.randn((N, 1), dtype=torch.float64, device="cuda", generator=g)
        for _ in range(steps):
            v = apply_Bt(apply_B(v / torch.linalg.norm(v)))
        return float(torch.sqrt(torch.linalg.norm(v)))

    def apply_h(h, x, trans=False):
        out = torch.empty_like(x)
        hb.hbs_apply(h, x, out, trans=trans)
        return out

    results = {}
    for i, mode in enumerate(modes):
        results[mode] = timed(mode, args.steps, args.warmup, sample_clocks=(i == 0))
    head = modes[0]
    res = results[head]
    nA = None
    if not args.no_accuracy:                     # Section 5 accuracy: 20 power steps on B^* B
        nA = power_norm(lambda x: A @ x, lambda x: A.T @ x)
        for mode, rr in results.items():
            h = rr["h"]
            rr["rel_error"] = power_norm(lambda x: apply_h(h, x) - A @ x,
                                         lambda x: apply_h(h, x, True) - A.T @ x) / nA
        if "fp64" in results:
            h0 = results["fp64"]["h"]
            n0 = power_norm(lambda x: apply_h(h0, x), lambda x: apply_h(h0, x, True))
            for mode, rr in results.items():
                if mode == "fp64":
                    continue
                h = rr["h"]
                rr["vs_fp64"] = power_norm(lambda x: apply_h(h, x) - apply_h(h0, x),
                                           lambda x: apply_h(h, x, True) - apply_h(h0, x, True)) / n0

    # end to end through the C ABI with host buffers: A in, factors out, every step
    e2e = None
    if not args.no_e2e:
        h = res["h"]
        cfg = MODES[head]
        src = A if cfg["a"] == "f64" else A32
        host_info = gpu_host_numa(gpu_id)
        with numa_local(host_info):                 # pinned pages on the GPU's own memory node
            A_host = torch.empty(src.shape, dtype=src.dtype, pin_memory=True)
            A_host.copy_(src)
            F_host = torch.empty(hb.hbs_factor_bytes(h), dtype=torch.uint8, pin_memory=True)
        dst = src                                   # the device copy the step multiplies
        streamed = cfg["sample"] == 0               # FP64 products take the pinned A directly

        def e2e_step(k=None, step=res["step"]):
            if streamed:                            # row blocks copied under the products
                step(A_src=A_host)
            else:
                dst.copy_(A_host, non_blocking=True)
                step()
            hb.hbs_copy_factors(h, F_host)

        e2e_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            e2e_step(k)
        e1.record(stream)
        barrier()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3)
        # the copies alone: all of A host -> device, and the factors device -> host
        c = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        c[0].record(stream)
        dst.copy_(A_host, non_blocking=True)
        c[1].record(stream)
        hb.hbs_copy_factors(h, F_host)
        c[2].record(stream)
        barrier()
        h2d_ms, d2h_ms = c[0].elapsed_time(c[1]), c[1].elapsed_time(c[2])
        # the products of the same steps alone, between events (the plain calls)
        for k in range(res["plain_steps"]):
            e2e_step(step=lambda A_src=None, k=k: res["plain_step"](k, A_src=A_src))
        torch.cuda.synchronize()
        streamed_products_ms = res["products_ms"]()          # both products, per e2e step
        a_bytes = src.numel() * src.element_size()
        e2e_ms = te / args.steps * 1e3
        dev_ms = res["elapsed"] / args.steps * 1e3
        e2e = {"value": world * N * s * args.steps / te, "unit": UNIT,
               "ms_per_step": e2e_ms, "device_ms_per_step": dev_ms,
               "overhead_ms_per_step": e2e_ms - dev_ms,
               "h2d_ms_all_of_A": h2d_ms, "h2d_gbs": a_bytes / h2d_ms / 1e6,
               "products_ms_per_step": streamed_products_ms,
               "products_ms_per_step_device_A": 2 * res["per_launch"] * 1e3,
               "d2h_ms_factors": d2h_ms, "d2h_gbs": hb.hbs_factor_bytes(h) / d2h_ms / 1e6,
               "host": {k: (len(v) if isinstance(v, list) else v) for k, v in host_info.items()},
               "a_transfer": "A streamed from pinned host memory by the library, copies overlapping "
                             "the products" if streamed else "A copied to the device before the call",
               "h2d_bytes_per_step": src.numel() * src.element_size(),
               "d2h_bytes_per_step": hb.hbs_factor_bytes(h)}

    value = world * N * s * args.steps / res["elapsed"]
    flops_product = 2.0 * N * N * s                          # one of the two products
    if MODES[head]["sample"] in (3, 4):
        pairs = 28 if MODES[head]["sample"] == 3 else 15
        peak = BF16_TFLOPS_SUSTAINED
        achieved = pairs * flops_product / res["per_launch"] / 1e12
        split = "oz_split_a" if pairs == 28 else "oz_split_shared"
        roofline = {"kernel": f"digit products per FP64 product ({split}, oz_split_b, oz_gemm, oz_reduce; "
                              f"{pairs} exact FP16 digit-pair products)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": f"bf16_tflops_sustained (of {PEAKS_SOURCE})"}
    elif MODES[head]["sample"] == 0:
        peak = SM_COUNT_GB300 * FP64_DFMA_PER_CLK_PER_SM * 2 * 2070e6 / 1e12
        achieved = flops_product / res["per_launch"] / 1e12
        roofline = {"kernel": "sample_gemm_f64 (Y = A Omega, Z = A^T Psi)", "bound": "alu",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": GEMM_READ_8192 * (N / 8192) ** 2 + GEMM_WRITE_8192 * (N / 8192),
                    "traffic_source": "ncu capture at N=8192: reads (A) scaled by (N/8192)^2, "
                                      "writes (split partials) by N/8192",
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
                    "probe_peak": peaks["fp64_probe"],
                    "probe_source": "hbs_probe_peaks: DFMA chains on every SM, measured in this run"}
    else:
        peak = BF16_TFLOPS_SUSTAINED
        achieved = 6 * flops_product / res["per_launch"] / 1e12
        roofline = {"kernel": "sliced_gemm_tc (bf16x6: 6 slice products per FP32 product)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": f"bf16_tflops_sustained (of {PEAKS_SOURCE})"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["elapsed"] / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "oz64": "f64 (exact FP16 digit products)", "mixed": "bf16x6/f32/f64",
                  "tc64": "bf16x6/f64", "cmp": "fp16 digits/df32/f64",
                  "mixed3": "bf16x3/f32/f64"}[head], "data": "synthetic",
        "config": {"workload": ("double-layer BIE" if args.workload == "doublelayer" else "log-kernel")
                               + f" N={N} r={r} s={s} leaf={leaf} dense",
                   "N": N, "r": r, "s": s, "leaf": leaf, "levels": L + 1, "mode": head,
                   "precision": MODES[head]["what"],
                   "l2": "inputs larger than L2 (A is %.1f GB, streamed every step)"
                         % (A.numel() * A.element_size() / 1e9),
                   "parallelism": f"replicas x{world}"},
        "rel_error": {"opnorm_power20": res.get("rel_error"), "vs": "dense A"},
        "compress_ms": res["elapsed"] / args.steps * 1e3,
        "sweep_gflop": sweep_flops(N, r, s, leaf) / 1e9,
        # per step: Philox draws + products (FP64: 2 GEMMs + 2 slice sums; bf16x6: 2 right-hand
        # splits + 2 GEMMs + 2 reductions; digits: 2 test-matrix splits + 1 A split + 2 GEMMs +
        # 2 reductions), then per tree level the side, bases, D and merge kernels (FP64: D in two
        # kernels; FP32: one)
        # (+ node_lq, the leaves' LQ, where the leaf height runs the one-CTA side form of an
        # FP64 sweep)
        "gpu_launches": args.steps * ({0: 2 + 2 + 2, 1: 2 + 6, 2: 2 + 6, 3: 2 + 3 + 4,
                                       4: 2 + 3 + 4}[MODES[head]["sample"]]
                                      + (1 if res["tuning"][0] > 0 and FINISH[MODES[head]["sweep"]] == "fp64"
                                         else 0)
                                      + sweep_launches(N, r, s, leaf, res["tuning"],
                                                       MODES[head]["sweep"] in (1, 2, 4))),
        "roofline": dict(roofline, sweep=res["sweep"]),
        "peaks": peaks,
        "clocks": res["clocks"],
        "step": "hbs_sample_execute: Philox draws, products and sweep in one call, the leaves' "
                "test-block LQ on a second stream while the products run (Section 1's single-view "
                "remark); plain_ms_per_step: hbs_draw_gaussian x2 + hbs_sample_products + "
                "hbs_execute, nothing overlapped",
        "modes": {m: {"ms_per_step": rr["elapsed"] / args.steps * 1e3,
                      "value": world * N * s * args.steps / rr["elapsed"],
                      "plain_ms_per_step": rr["elapsed_plain"] / rr["plain_steps"] * 1e3,
                      "overlap_saving_ms_per_step": (rr["elapsed_plain"] / rr["plain_steps"]
                                                     - rr["elapsed"] / args.steps) * 1e3,
                      "rel_error": rr.get("rel_error"), "vs_fp64": rr.get("vs_fp64"),
                      "products_ms_per_launch": rr["per_launch"] * 1e3,
                      "sweep_ms": rr["sweep"]["total"]["ms"],
                      "sweep_frac_by_kernel": {k: round(v["frac"], 3)
                                               for k, v in rr["sweep"]["per_kernel"].items()},
                      "tuned_row_slices": rr["tuning"],
                      "what": MODES[m]["what"]} for m, rr in results.items()},
    }
    if e2e:
        line["e2e"] = e2e
    if not args.only and args.workload == "logkernel" and (not args.no_batched or not args.no_config3
                                                            or not args.no_apply):
        for rr in results.values():
            rr["h"].free()
        results = {}
        del A, A32
        torch.cuda.empty_cache()
        if not args.no_config3:
            line["config3"] = run_config3(hb, torch, min(args.steps, 5), 3)
        if not args.no_batched:
            line["batched"] = run_batched(hb, torch)
        if not args.no_apply:
            line["apply"] = run_apply(hb, torch, logN=22, reps=3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, sample = oracle_sample_time(N, r, s, leaf, workload=args.workload)
        line["cpu_baseline"] = {"value": N * s / t_cpu, "unit": UNIT, "cores": cpu_cores(),
                                "kind": "oracle", "sample": sample}
    for rr in results.values():
        rr["h"].free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
