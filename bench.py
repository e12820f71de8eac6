"""Benchmark of one self-consistent GF2 iteration on one GB300 (per rank).

Workload: H32 finite lattice 2x4x4 at 2.0 bohr, 6-31G (N = 64 basis
functions, 32 electrons), beta = 100 Eh^-1, uniform tau grid with 4097 points,
8192 Matsubara frequencies; synthetic inputs built by ``gf2_inputs``
(closed-form integrals, RHF start).  One step = one pass over every row of the
hot path, all through the libgf2 C-ABI with inputs resident in HBM:

  tail moments -> G(i w) -> G(tau) -> Sigma(tau) [split BF16, tcgen05] ->
  Sigma damping -> Sigma(tau) -> Sigma(i w) -> mu search with the Dyson
  inverse -> Fock build -> Galitskii-Migdal energy.

Every step starts from the same state (HF Green's function, F_HF, mu_HF), so
the steps do identical work.  ``value`` = 8 N^5 n_tau useful Sigma flops per
step / step time (the Sigma-equivalent throughput of a whole iteration);
the Sigma build alone, the FP64 GPU path (timed on sampled tau points and
scaled) and a per-kernel breakdown are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x6|bf16x3|fp16x3|fp16x6]
  python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample
  python bench.py --workload batch   # batched Sigma(tau) over 24 systems, N = 4 .. 50
  python bench.py --workload h32_sto3g   # N = 32 lattice at 1.4 / 2.0 / 3.0 bohr: split vs FP64
  python bench.py --workload converge    # GF2 to convergence on the H10 chain, split vs FP64
  python bench.py --workload h64         # H64 lattice (N = 128), the 128-wide split Sigma
  python bench.py --workload sigma --n-bf 128 --n-tau 33   # the Sigma build alone (kernel profiles)
  python bench.py --workload h32_df      # density-fitted integrals (m = 192) on the power mesh

The batch workload has the sizes of a multi-system study: linear H_n chains,
n = 4, 6, ..., 20, 24, 28, ..., 44, 50 (STO-3G, N = n) plus eight H32 2x4x4
STO-3G lattices (N = 32), each with n_tau = 2049.  Its inputs are seeded random
symmetric G(tau) and 8-fold-symmetric integrals of those sizes (the Sigma
build's cost does not depend on the values); one step is one
gf2_sigma_tau_batched call over all 24 systems (a replay of the recorded graph).
"""

import argparse
import hashlib
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

WORKLOAD = {"name": "h32_lattice_631g", "lattice": "2x4x4", "spacing_bohr": 2.0, "basis": "6-31g",
            "n_bf": 64, "n_elec": 32, "beta": 100.0, "n_tau": 4097, "n_iw": 8192}
METRIC = "Σ(τ) s/iter & TFLOP/s at N=64: split-BF16 vs FP64 GPU path, |ΔE|≤1µEh"
PRECS = {"bf16x3": 1, "bf16x6": 2, "fp16x3": 3, "fp16x6": 4, "fp64": 0}
ISSUED = {"bf16x3": 3, "bf16x6": 6, "fp16x3": 3, "fp16x6": 6}   # split products per useful multiply


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x6", choices=sorted(ISSUED))
    ap.add_argument("--fp64-points", type=int, default=8, help="tau points for the FP64 path timing")
    ap.add_argument("--no-energy-check", action="store_true")
    ap.add_argument("--cpu-points", type=int, default=48, help="tau points of the oracle CPU baseline sample")
    ap.add_argument("--ref-points", type=int, default=4, help="tau points per step of --impl reference")
    ap.add_argument("--n-tau", type=int, default=None, help="override the tau grid (smaller cases for ncu)")
    ap.add_argument("--n-iw", type=int, default=None, help="override the frequency count")
    ap.add_argument("--workload", default="h32_631g",
                    choices=["h32_631g", "h64", "batch", "h32_sto3g", "converge", "sigma", "h32_mesh", "h64_mesh",
                             "h32_df"])
    ap.add_argument("--n-bf", type=int, default=128, help="basis size of --workload sigma")
    ap.add_argument("--mesh", type=int, nargs=2, default=(7, 32), metavar=("P", "U"),
                    help="power mesh of --workload h32_mesh / h64_mesh (P halvings, U steps per interval)")
    ap.add_argument("--max-outer", type=int, default=30, help="outer GF2 iterations of --workload converge")
    ap.add_argument("--profile-run", action="store_true",
                    help="warm-up and timed steps only (no e2e, FP64 sample, energy check or CPU baseline)")
    args = ap.parse_args()
    if args.n_tau:
        WORKLOAD["n_tau"] = args.n_tau
    if args.n_iw:
        WORKLOAD["n_iw"] = args.n_iw
    return args


# --------------------------------------------------------------------------- setup

def build_inputs():
    import gf2_inputs as gi
    s = gi.build_system(WORKLOAD["name"], spacing=WORKLOAD["spacing_bohr"])
    r = gi.rhf(s)
    return s, r


def dist_setup(n):
    if n <= 1:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(n)))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, world, dist


def max_over_ranks(x, dist):
    """The largest per-rank time (the whole job is as slow as its slowest replica)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = str(device_index)
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"gf2_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        loaded = [sm for sm, _, _ in rows] or [0.0]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx for _, mx, _ in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def peak_label(kind, what):
    """Where a roofline denominator came from."""
    if kind == "measured":
        return f"measured {what} (MEASURED_PEAKS.json)"
    return f"fallback {what} (no MEASURED_PEAKS.json: an earlier GB300 measurement)"


def ncu_traffic(kernel, prec="bf16x6"):
    """DRAM bytes per launch of `kernel` (captured in precision `prec`) from the
    committed ncu summary, if the kernel source has not changed since."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel if prec == "bf16x6" else f"{kernel}@{prec}")
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != d["source_sha256"]:
        return None
    return d["dram_bytes_per_launch"]


def load_golden(n_tau, n_iw):
    """The oracle's first step on this workload's grid, if the fixture exists."""
    p = os.path.join(ROOT, "tests", "golden", f"h32_631g_first_step_t{n_tau}_w{n_iw}.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    d["_file"] = os.path.relpath(p, ROOT)
    return d


# --------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, dist):
    import torch
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    s, r = build_inputs()
    N, n_tau, n_iw, beta = s.nbf, WORKLOAD["n_tau"], WORKLOAD["n_iw"], WORKLOAD["beta"]
    prec = PRECS[args.prec]
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    S, hcore, F0 = f64(s.S), f64(s.h), f64(r.F)
    ctx = g.Context(N, n_tau, n_iw, beta)
    h = ctx.handle
    g.gf2_set_integrals(h, f64(s.eri))
    g.gf2_set_overlap(h, S)
    # state of the first GF2 iteration: finite-temperature HF Green's function
    G_iw0 = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
    P0 = torch.zeros(N, N, dtype=torch.float64, device="cuda")
    mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G_iw0, P0)

    moments = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
    G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_new = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_tau = torch.zeros(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
    sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
    G_iw = torch.empty_like(G_iw0)
    P = torch.empty_like(P0)
    F_new = torch.empty_like(F0)
    damping = 1.0
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(G_in, F_in, out, sigma_events=None):
        g.gf2_tail_moments(h, S, F_in, mu_hf, None, moments)                 # tail moments
        g.gf2_fft_iw_to_tau(h, G_in, moments, G_tau)                         # G(i w) -> G(tau)
        if sigma_events:
            sigma_events[0].record(stream)
        g.gf2_sigma_tau(h, G_tau, Sig_new, prec)                             # Sigma(tau)
        if sigma_events:
            sigma_events[1].record(stream)
        g.gf2_combine(h, [damping, 1.0 - damping], [Sig_new, Sig_tau], Sig_tau)  # damping
        g.gf2_fft_tau_to_iw(h, Sig_tau, Sig_iw, sig12)                       # Sigma(tau) -> Sigma(i w)
        mu, nev = g.gf2_mu_search(h, S, F_in, Sig_iw, sig12, s.n_elec, mu_hf, G_iw, P)  # mu + Dyson
        g.gf2_fock(h, hcore, P, F_new)                                       # Fock
        e1, e2 = g.gf2_energy(h, hcore, F_in, P, S, G_iw, Sig_iw, sig12)      # energy
        out.append((s.e_nuc + e1 + e2, mu, nev))

    log = []
    for _ in range(args.warmup):
        step(G_iw0, F0, log)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # the timed steps run without the per-launch event profiler (its events would
    # sit inside the timed region); the launch count is kept either way.  The
    # --profile-run mode (ncu launch lists) profiles the timed steps themselves.
    g.gf2_profile(h, bool(args.profile_run))
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0, t1 = ev(), ev()
    sig_ev = [(ev(), ev()) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.steps):
        step(G_iw0, F0, log, sig_ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof, launches = g.gf2_profile_report(h)
    g.gf2_profile(h, False)
    if not args.profile_run:
        # per-kernel times from the same number of extra, profiled steps
        g.gf2_profile(h, True)
        for _ in range(args.steps):
            step(G_iw0, F0, log)
        torch.cuda.synchronize()
        prof, _ = g.gf2_profile_report(h)
        g.gf2_profile(h, False)
    ms_total = t0.elapsed_time(t1)
    ms_step = ms_total / args.steps
    sigma_ms = statistics.mean(a.elapsed_time(b) for a, b in sig_ev)
    ms_step = max_over_ranks(ms_step, dist)
    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms_step, "sigma_ms": sigma_ms,
                              "kernels": {k: v for k, v in prof.items()}, "launches": launches}))
        ctx.close()
        return

    # end to end: host buffers in, host scalars and P out, copies inside the timed
    # region.  Every step's G(i w) and F come from pinned host memory; the copy of
    # step k+1's inputs runs on a copy stream into the other of two device
    # buffers while step k computes (it waits until step k-1 has released that
    # buffer), and step k waits for its own copy.
    G_host = G_iw0.cpu().pin_memory()
    F_host = F0.cpu().pin_memory()
    P_host = torch.empty(N, N, dtype=torch.float64).pin_memory()
    G_dev = [torch.empty_like(G_iw0) for _ in range(2)]
    F_dev = [torch.empty_like(F0) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [ev(), ev()]
    released = [ev(), ev()]
    used = [False, False]

    def issue_copy(buf):
        if used[buf]:
            copy_stream.wait_event(released[buf])
        with torch.cuda.stream(copy_stream):
            G_dev[buf].copy_(G_host, non_blocking=True)
            F_dev[buf].copy_(F_host, non_blocking=True)
            copied[buf].record(copy_stream)

    e2e_steps = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    copy_stream.wait_event(a)
    issue_copy(0)
    for k in range(e2e_steps):
        cur = k % 2
        if k + 1 < e2e_steps:
            issue_copy(1 - cur)
        stream.wait_event(copied[cur])
        step(G_dev[cur], F_dev[cur], log)
        released[cur].record(stream)
        used[cur] = True
        P_host.copy_(P, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e2e_steps
    h2d = G_host.numel() * 16 + F_host.numel() * 8
    d2h = P_host.numel() * 8 + 3 * 8

    # FP64 GPU path on sampled points, and split vs FP64 on the same points
    flops_tau = 8.0 * N ** 5
    pts = np.linspace(1, n_tau - 2, args.fp64_points).astype(int)
    k0 = int(pts[0])
    cnt = args.fp64_points
    out64 = torch.empty(cnt, N, N, dtype=torch.float64, device="cuda")
    g.gf2_sigma_tau_points(h, G_tau, k0, cnt, out64, 0)  # warm
    torch.cuda.synchronize()
    a.record(stream)
    g.gf2_sigma_tau_points(h, G_tau, k0, cnt, out64, 0)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_ms_per_tau = a.elapsed_time(b) / cnt
    outs = torch.empty_like(out64)
    g.gf2_sigma_tau_points(h, G_tau, k0, cnt, outs, prec)
    rel = ((outs - out64).abs().max() / out64.abs().max()).item()

    energy_check = None
    if not args.no_energy_check:
        # E of the first GF2 iteration with the FP64 GPU Sigma vs the split Sigma
        g.gf2_sigma_tau(h, G_tau, Sig_new, 0)
        g.gf2_fft_tau_to_iw(h, Sig_new, Sig_iw, sig12)
        G64 = torch.empty_like(G_iw)
        P64 = torch.empty_like(P)
        mu64, _ = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, G64, P64)
        e1, e2 = g.gf2_energy(h, hcore, F0, P64, S, G64, Sig_iw, sig12)
        e64 = s.e_nuc + e1 + e2
        energy_check = {"E_split": log[-1][0], "E_fp64_gpu": e64, "abs_dE": abs(log[-1][0] - e64),
                        "max_abs_dP": (P - P64).abs().max().item(), "mu_split": log[-1][1], "mu_fp64": mu64,
                        "n_split": float(torch.trace(P @ S)), "n_fp64": float(torch.trace(P64 @ S))}

    # the same step against the oracle's values for it (stored fixture, written by
    # tests/golden/make_h32_631g_first_step.py from oracle/ only)
    golden = load_golden(n_tau, n_iw)
    oracle_check = None
    if golden is not None:
        P_or = torch.as_tensor(np.array(golden["P"]), device="cuda")
        oracle_check = {"fixture": golden["_file"], "E_oracle": golden["E"],
                        args.prec: {"abs_dE": abs(log[-1][0] - golden["E"]),
                                    "max_abs_dP": (P - P_or).abs().max().item()}}
        if energy_check:
            oracle_check["fp64_gpu"] = {"abs_dE": abs(energy_check["E_fp64_gpu"] - golden["E"]),
                                        "max_abs_dP": (P64 - P_or).abs().max().item()}

    # the other split precisions on the same state: Sigma build time and the same checks
    alternates = {}
    for name in ([] if args.no_energy_check else [x for x in ("fp16x3", "bf16x3") if x != args.prec]):
        pc = PRECS[name]
        g.gf2_sigma_tau(h, G_tau, Sig_new, pc)
        torch.cuda.synchronize()
        times = []
        for _ in range(3):
            a.record(stream)
            g.gf2_sigma_tau(h, G_tau, Sig_new, pc)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        g.gf2_fft_tau_to_iw(h, Sig_new, Sig_iw, sig12)
        Ga, Pa = torch.empty_like(G_iw), torch.empty_like(P)
        mua, _ = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, Ga, Pa)
        e1, e2 = g.gf2_energy(h, hcore, F0, Pa, S, Ga, Sig_iw, sig12)
        g.gf2_sigma_tau_points(h, G_tau, k0, cnt, outs, pc)
        if oracle_check is not None:
            oracle_check[name] = {"abs_dE": abs(s.e_nuc + e1 + e2 - golden["E"]),
                                  "max_abs_dP": (Pa - P_or).abs().max().item()}
        alternates[name] = {"sigma_s_per_iter": statistics.median(times) * 1e-3,
                            "sigma_tflops_useful": flops_tau * n_tau / (statistics.median(times) * 1e-3) / 1e12,
                            "issued_products": ISSUED[name],
                            "split_vs_fp64_max_rel_err": ((outs - out64).abs().max() / out64.abs().max()).item(),
                            "abs_dE_vs_fp64_gpu": abs(s.e_nuc + e1 + e2 - e64) if energy_check else None,
                            "max_abs_dP": (Pa - P64).abs().max().item() if energy_check else None}

    # one full-frequency Dyson sweep on its own, for its roofline
    G_dy = torch.empty_like(G_iw)
    g.gf2_dyson(h, mu_hf, S, F0, Sig_iw, G_dy)
    torch.cuda.synchronize()
    dy = []
    for _ in range(3):
        a.record(stream)
        g.gf2_dyson(h, mu_hf, S, F0, Sig_iw, G_dy)
        b.record(stream)
        torch.cuda.synchronize()
        dy.append(a.elapsed_time(b))
    dyson_ms = statistics.median(dy)
    del G_dy

    hbm_gbs, bf16_burst, bf16_sust, peak_kind = measured_peaks()
    useful = flops_tau * n_tau
    value = useful / (ms_step * 1e-3) / 1e12 * world
    sigma_tflops = useful / (sigma_ms * 1e-3) / 1e12

    # dominant kernel and its roofline
    steps = args.steps
    per_kernel = {k: {"launches": c, "ms_per_step": ms / steps} for k, (c, ms) in prof.items()}
    issued_factor = ISSUED[args.prec]
    C = 32
    n4 = float(N) ** 4
    # per launch (one chunk of C time points for the Sigma stages): the stage's
    # useful flops (its algorithmic work; the split products issued per useful
    # multiply divide the BF16 peak), and the bytes of the stage's own FP32
    # intermediates (T2 written by stages 1+2, T2 read and T3 written by stage 3,
    # T3 read by stage 4), reported beside the roofline as implementation traffic.
    # with the pair symmetry (im|qk) = (qk|im) of v the sandwich computes only the
    # unique (i, q) tiles of the stage-2 intermediate (1056 of 2048 units per pair
    # of time points) and mirrors the rest: its work is counted as computed
    pair_sym = bool(np.abs(s.eri - s.eri.transpose(2, 3, 0, 1)).max() <= 1e-12 * np.abs(s.eri).max())
    sym_frac = 1056.0 / 2048.0 if pair_sym else 1.0
    exec_frac = (4.0 * sym_frac + 4.0) / 8.0  # share of the 8 N^5 flops per point the kernels execute
    tensor_work = {"sigma_sandwich": (4.0 * N ** 5 * C * sym_frac, 4.0 * n4 * C),
                   "sigma_xform": (2.0 * N ** 5 * C, 8.0 * n4 * C),
                   "sigma_contract": (2.0 * N ** 5 * C, 4.0 * n4 * C)}
    # kernels whose every launch covers the full problem (per-launch averages are
    # exact), as (FP64 flops, bytes): the transforms run one M-point FFT per
    # matrix element (5 M log2 M flops) and read one grid and write the other;
    # the energy reads G(i w) and Sigma(i w) (Re G_ij Sigma_ji: 2 flops); the
    # Fock build reads v once with two multiply-adds per element
    M = n_tau - 1
    fft_flops = 5.0 * M * math.log2(M) * N * N
    other_work = {
        "fft_iw_to_tau": (fft_flops, n_iw * N * N * 16 + n_tau * N * N * 8),
        "fft_tau_to_iw": (fft_flops, n_iw * N * N * 16 + n_tau * N * N * 8),
        "energy_reduce": (2.0 * n_iw * N * N, n_iw * N * N * 32),
        "fock_build": (4.0 * n4, 8.0 * n4),
    }
    fp64_peak = 1.25 * (clocks["sm_mhz"] / 2070.0 if clocks else 1.0)
    split_peak = bf16_sust / issued_factor

    def roofline_of(k):
        n_launch, k_ms = prof[k]
        dur = k_ms / n_launch * 1e-3
        if k in tensor_work:
            # a Sigma stage's algorithmic work is its useful flops (2 N^5 per time
            # point per contraction); its FP32 intermediates are the implementation's
            # own traffic and are reported beside it (stage_io_gbs, traffic)
            flops, nbytes = tensor_work[k]
            bound, achieved, peak, unit = "tensor", flops / dur / 1e12, split_peak, "TFLOP/s"
            src = (peak_label(peak_kind, f"sustained BF16 {bf16_sust} TFLOP/s") +
                   f" / {issued_factor} split products per useful flop")
        else:
            # the roof reached first: FP64 flops at the FP64 peak or bytes at the copy bandwidth
            flops, nbytes = other_work.get(k, (float("nan"), float("nan")))
            if flops / (fp64_peak * 1e12) > nbytes / (hbm_gbs * 1e9):
                bound, achieved, peak, unit = "alu", flops / dur / 1e12, fp64_peak, "TFLOP/s"
                src = "derived: 1.25 TFLOP/s FP64 nominal at 2070 MHz, scaled to the sampled clock"
            else:
                bound, achieved, peak, unit = "hbm", nbytes / dur / 1e9, hbm_gbs, "GB/s"
                src = peak_label(peak_kind, f"HBM copy {hbm_gbs} GB/s")
        traffic = ncu_traffic(k, args.prec)
        r = {"kernel": k, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
             "frac": achieved / peak, "traffic": traffic, "peak_source": src, "ms_per_launch": dur * 1e3}
        if k in tensor_work:
            r["algorithmic_flops_per_launch"] = flops
            r["issued_frac_of_bf16"] = flops * issued_factor / dur / 1e12 / bf16_sust
            r["stage_io_bytes_per_launch"] = nbytes
            r["stage_io_gbs"] = nbytes / dur / 1e9
            r["stage_io_frac_of_hbm"] = nbytes / dur / 1e9 / hbm_gbs
            if traffic:
                r["traffic_gbs"] = traffic / dur / 1e9
        return r

    dom = max(prof, key=lambda k: prof[k][1])
    sigma_rooflines = {k: roofline_of(k) for k in tensor_work if k in prof}
    other_rooflines = {k: roofline_of(k) for k in other_work if k in prof}
    # Dyson: the mu search mixes full and coarse (n_iw/8) launches, so a full
    # sweep is timed on its own; a complex symmetric inverse needs N^3/2 complex
    # multiply-adds (4 N^3 flops) per frequency
    dyson_flops = 4.0 * N ** 3 * n_iw
    other_rooflines["dyson_inverse"] = {
        "kernel": "dyson_inverse", "bound": "alu", "achieved": dyson_flops / (dyson_ms * 1e-3) / 1e12,
        "peak": fp64_peak, "unit": "TFLOP/s", "frac": dyson_flops / (dyson_ms * 1e-3) / 1e12 / fp64_peak,
        "traffic": None, "ms_per_launch": dyson_ms,
        "peak_source": "derived: 1.25 TFLOP/s FP64 nominal at 2070 MHz, scaled to the sampled clock",
        "sample": f"one full sweep over {n_iw} frequencies, median of 3"}
    roofline = {**sigma_rooflines, **other_rooflines}.get(dom) or roofline_of(dom)
    # the tensor kernels together
    tc_ms = sum(prof.get(k, (0, 0.0))[1] for k in ("sigma_sandwich", "sigma_xform", "sigma_contract")) / steps

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic (closed-form s-Gaussian integrals, RHF start)",
        "config": config_of(world),
        "sigma": {"s_per_iter": sigma_ms * 1e-3, "tflops_useful": sigma_tflops,
                  "stage2_pair_symmetry": pair_sym,
                  "tensor_kernels_ms": tc_ms,
                  # split products the kernels execute (the pair symmetry skips part of
                  # stages 1+2), against the sustained BF16 peak: over the whole build
                  # (including its FP64 basis transforms) and over the three tensor kernels
                  "executed_share_of_8n5": exec_frac,
                  "tflops_issued": sigma_tflops * exec_frac * issued_factor,
                  "issued_frac_of_bf16_build": sigma_tflops * exec_frac * issued_factor / bf16_sust,
                  "issued_frac_of_bf16_tensor_kernels": (useful * exec_frac * issued_factor / (tc_ms * 1e-3) / 1e12
                                                         / bf16_sust if tc_ms > 0 else None),
                  # the same with every useful flop of Eq. Sigma counted (8 N^5 per point):
                  # the products a build without the symmetry would issue in this time
                  "useful_equiv_frac_of_bf16_build": sigma_tflops * issued_factor / bf16_sust},
        "fp64_gpu_path": {"sigma_s_per_iter": fp64_ms_per_tau * 1e-3 * n_tau,
                          "tflops": flops_tau / (fp64_ms_per_tau * 1e-3) / 1e12,
                          "sample": f"{cnt} tau points from k={k0}",
                          "split_vs_fp64_max_rel_err": rel},
        "speedup_split_vs_fp64_sigma": fp64_ms_per_tau * n_tau / sigma_ms,
        "alternate_precisions": alternates,
        "mu_evaluations_per_step": log[-1][2],
        "kernels": per_kernel,
        "roofline": roofline,
        "sigma_rooflines": sigma_rooflines,
        "other_rooflines": other_rooflines,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": useful / (e2e_ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(s, r, args)
        # the accuracy checks go last, where a reader of the end of the line finds them
        line["energy_check"] = energy_check
        line["oracle_check"] = oracle_check
        print(json.dumps(line))
    ctx.close()


# --------------------------------------------------------------------------- oracle (CPU)

def oracle_setup(s, r):
    """Untimed inputs of the oracle sample: the finite-temperature HF Green's
    function G(i w) at mid-gap mu on every frequency (the state a step starts
    from) and its tail moments."""
    from oracle import dyson as od
    from oracle import transforms as ot
    from oracle import sigma as osg

    beta, n_iw = WORKLOAD["beta"], WORKLOAD["n_iw"]
    mu = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    return {"mu": mu, "G_iw": od.dyson(mu, s.S, r.F, None, beta, n_iw), "mom": ot.tail_moments(s.S, r.F, mu),
            "W": osg.exchange_combination(s.eri)}


def oracle_sample(s, r, setup, n_points):
    """The oracle (as it stands) on a fixed fraction phi = n_points / n_tau of
    one GF2 step, every row cut to that fraction of its units:
      G(tau) at n_points grid points (pairs k, M - k) by the direct sum over all
      n_iw frequencies; Eq. Sigma at those points; Sigma(tau) -> Sigma(i w) on
      phi * n_iw frequencies (cubic-interpolant weights over all n_tau points;
      the points not computed here carry copies of computed ones); the
      bisection mu search on those frequencies (the oracle's own evaluation
      count); the energy sum on them; plus one whole Fock build and the tail
      moments (both O(N^4) or less).  Returns (measured seconds, detail)."""
    from oracle import dyson as od
    from oracle import energy as oe
    from oracle import sigma as osg
    from oracle import transforms as ot
    from oracle.fock import fock

    N, n_tau, n_iw, beta = s.nbf, WORKLOAD["n_tau"], WORKLOAD["n_iw"], WORKLOAD["beta"]
    M = n_tau - 1
    half = max(1, n_points // 2)
    ks = np.linspace(1, M // 2 - 1, half).astype(int)
    taus = np.concatenate([ks, M - ks])
    nw = max(4, int(round(n_iw * len(taus) / n_tau)))
    rows = {}
    t_all = time.perf_counter()
    t = time.perf_counter()
    mom = ot.tail_moments(s.S, r.F, setup["mu"])
    G_pts = ot.iw_to_tau(setup["G_iw"], mom, beta, n_tau, taus=taus)
    rows["iw_to_tau_s"] = time.perf_counter() - t
    t = time.perf_counter()
    sig = np.array([osg.sigma_factored(G_pts[j], -G_pts[(j + half) % len(taus)], s.eri, setup["W"])
                    for j in range(len(taus))])
    rows["sigma_s"] = time.perf_counter() - t
    t = time.perf_counter()
    grid = np.resize(sig, (n_tau, N, N))
    Sig_iw = ot.tau_to_iw(grid, beta, nw)
    sig1, sig2 = ot.sigma_expansion(grid, beta)
    rows["tau_to_iw_s"] = time.perf_counter() - t
    t = time.perf_counter()
    mu, G, P, nev = od.mu_search(s.S, r.F, Sig_iw, sig1, sig2, s.n_elec, beta, nw)
    rows["mu_search_s"] = time.perf_counter() - t
    t = time.perf_counter()
    fock(s.h, s.eri, P)
    oe.e_one_body(P, s.h, r.F) + oe.e_two_body(G, Sig_iw, sig1, s.S, beta)
    rows["fock_energy_s"] = time.perf_counter() - t
    total = time.perf_counter() - t_all
    detail = {"tau_points": int(len(taus)), "frequencies": nw, "fraction_of_step": len(taus) / n_tau,
              "mu_evaluations": int(nev), "rows_s": rows}
    return total, detail


def _sample_text(detail):
    return (f"the oracle on {detail['fraction_of_step']:.4f} of one step, every row cut to that fraction: "
            f"G(tau) and Eq. Sigma at {detail['tau_points']} of {WORKLOAD['n_tau']} time points, "
            f"Sigma(tau)->Sigma(iw), the bisection mu search ({detail['mu_evaluations']} Dyson evaluations) "
            f"and the energy sum on {detail['frequencies']} of {WORKLOAD['n_iw']} frequencies, one whole "
            f"Fock build (the tail subtraction over all frequencies and the Fock build are not cut, so the "
            f"sample is slightly more than that fraction); value = Sigma-equivalent flops of that fraction "
            f"(8 N^5 per time point) / measured time")


def oracle_full_iteration_h10():
    """One whole outer GF2 iteration of the oracle, measured, on a workload it
    finishes in seconds: the H10 chain (STO-3G, 1.8 bohr, beta = 100, n_tau =
    2049, n_iw = 4096) from its converged HF state: tail moments, G(i w) ->
    G(tau), Eq. Sigma at every time point, Sigma(tau) -> Sigma(i w), the inner
    loop (mu searches and Fock rebuilds) to |R| < 1e-8, the energy."""
    import gf2_inputs as gi
    from oracle import gf2 as og
    s = gi.build_system("h10_chain_sto3g")
    r = gi.rhf(s)
    beta, n_tau, n_iw = 100.0, 2049, 4096
    F, mu, G, P = og.inner_loop(s, r.F, None, None, None, beta, n_iw)
    st = og.GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F), sig2=np.zeros_like(F))
    t = time.perf_counter()
    _, Sig_tau = og.self_energy_step(s, st, beta, n_tau, n_iw)
    Sig_iw, sig1, sig2 = og.sigma_to_iw(Sig_tau, beta, n_iw)
    st.F, st.mu, st.G_iw, st.P = og.inner_loop(s, F, Sig_iw, sig1, sig2, beta, n_iw)
    st.Sigma_iw, st.sig1 = Sig_iw, sig1
    E = og.energy(s, st, beta)[0]
    return {"workload": f"H10 chain 1.8 bohr, STO-3G (N=10), beta={beta}, n_tau={n_tau}, n_iw={n_iw}",
            "step": "one outer GF2 iteration from the HF state, every row, inner loop to |R| < 1e-8",
            "measured_s": time.perf_counter() - t, "E": E, "cores": _cores()}


def cpu_baseline(s, r, args):
    setup = oracle_setup(s, r)
    total, detail = oracle_sample(s, r, setup, args.cpu_points)
    useful = 8.0 * s.nbf ** 5 * detail["tau_points"]
    return {"value": useful / total / 1e12, "unit": "TFLOP/s", "cores": _cores(), "kind": "oracle",
            "sample": _sample_text(detail), "measured_s": total,
            "estimated_s_per_iter": total / detail["fraction_of_step"], "estimated": True, "detail": detail,
            "full_iteration_measured": oracle_full_iteration_h10()}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def config_of(world):
    return {"workload": (f"H32 lattice 2x4x4 at 2.0 bohr, 6-31G (N=64), beta=100, "
                         f"n_tau={WORKLOAD['n_tau']}, n_iw={WORKLOAD['n_iw']}"),
            "step": "one GF2 outer iteration, all hot-path rows",
            "l2": "inputs larger than L2 (G(iw) 537 MB, intermediates 6 GB)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world, dist):
    if rank != 0:
        return
    s, r = build_inputs()
    setup = oracle_setup(s, r)
    for _ in range(args.warmup):
        oracle_sample(s, r, setup, 2)
    times, detail = [], None
    for _ in range(args.steps):
        total, detail = oracle_sample(s, r, setup, args.ref_points)
        times.append(total)
    t_step = statistics.mean(times)
    useful = 8.0 * s.nbf ** 5 * detail["tau_points"]
    value = useful / t_step / 1e12
    cfg = config_of(world)  # the same workload as the GPU arm; the CPU sample is described in step_is
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "step_is": ("a bounded sample: " + _sample_text(detail)),
            "estimated_s_per_iter": t_step / detail["fraction_of_step"], "estimated": True,
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": _cores(), "kind": "oracle",
                             "sample": _sample_text(detail)},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "detail": detail}
    print(json.dumps(line))


BATCH_SIZES = [4, 6, 8, 10, 12, 14, 16, 18, 20, 24, 28, 32, 36, 40, 44, 50] + [32] * 8
BATCH_N_TAU = 2049


def run_batch(args, rank, world, dist):
    """Batched Sigma(tau) over the 24 systems of the multi-system workload."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prec = PRECS[args.prec]
    sizes, n_tau = BATCH_SIZES, BATCH_N_TAU
    Gs = [torch.as_tensor(gi.random_symmetric_g(n, n_tau, seed=500 + i), device="cuda") for i, n in enumerate(sizes)]
    outs = [torch.empty_like(x) for x in Gs]
    useful = sum(8.0 * n ** 5 * n_tau for n in sizes)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(p, steps, warmup):
        b = g.Batch(sizes, [n_tau] * len(sizes))
        for i, n in enumerate(sizes):
            g.gf2_batch_set_system(b.handle, i, torch.as_tensor(gi.random_eri(n, seed=600 + i), device="cuda"))
        t = time.perf_counter()
        g.gf2_batch_tune(b.handle, Gs, p)
        tune_s = time.perf_counter() - t
        plan = [g.gf2_batch_plan(b.handle, i) + (g.gf2_batch_partner(b.handle, i),) for i in range(len(sizes))]
        for _ in range(warmup):
            g.gf2_sigma_tau_batched(b.handle, Gs, outs, p)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        a, c = ev(), ev()
        a.record(stream)
        for _ in range(steps):
            g.gf2_sigma_tau_batched(b.handle, Gs, outs, p)
        c.record(stream)
        torch.cuda.synchronize()
        b.close()
        return a.elapsed_time(c) / steps, tune_s, plan

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, tune_s, plan = timed(prec, args.steps, args.warmup)
    clocks = sampler.stop()
    ms64, _, _ = timed(PRECS["fp64"], 1, 1)
    ms = max_over_ranks(ms, dist)
    names = {0: "fp64", 1: "bf16x3", 2: "bf16x6", 3: "fp16x3", 4: "fp16x6"}
    line = {"metric": "batched Σ(τ) build: useful TFLOP/s over 24 systems of uneven N", "value":
            useful / (ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic (seeded random G(tau) and integrals)",
            "config": {"workload": "24 systems: H_n chains n=4..50 (16) + 8 H32 lattices, STO-3G sizes, n_tau=2049",
                       "step": "one gf2_sigma_tau_batched call (graph replay)", "parallelism": f"replicas x{world}",
                       "l2": "inputs 1.0 GB, intermediates of the split instances several GB"},
            "all_fp64_ms_per_step": ms64, "speedup_vs_all_fp64": ms64 / ms, "tune_s": tune_s,
            "plan": [{"N": n, "path": names[p], "est_ms": round(e, 3), "lane": l, "slots_per_launch": c,
                      "shares_tiles_with": q}
                     for n, (p, e, l, c, q) in zip(sizes, plan)],
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))


def run_h32_sto3g(args, rank, world, dist):
    """H32 2x4x4 STO-3G lattice (N = 32) at three spacings: the first GF2
    iteration from the finite-temperature HF state with the FP64 and the split
    Sigma builds; Sigma seconds per iteration and the energy / density error of
    each split precision against the FP64 GPU path."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n_tau, n_iw, beta = 4097, 8192, 100.0
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    rows = []
    for a in (1.4, 2.0, 3.0):
        s = gi.build_system("h32_lattice_sto3g", spacing=a)
        r = gi.rhf(s)
        N = s.nbf
        ctx = g.Context(N, n_tau, n_iw, beta)
        h = ctx.handle
        S, hc, F0 = f64(s.S), f64(s.h), f64(r.F)
        g.gf2_set_integrals(h, f64(s.eri))
        g.gf2_set_overlap(h, S)
        G_iw = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
        P = torch.zeros(N, N, dtype=torch.float64, device="cuda")
        mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
        mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G_iw, P)
        mom = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
        G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
        g.gf2_tail_moments(h, S, F0, mu_hf, None, mom)
        g.gf2_fft_iw_to_tau(h, G_iw, mom, G_tau)
        row = {"spacing_bohr": a}
        ref = None
        for name in ("fp64", "bf16x3", "fp16x3", "bf16x6"):
            pc = PRECS[name]
            Sig = torch.empty_like(G_tau)
            g.gf2_sigma_tau(h, G_tau, Sig, pc)
            t0, t1 = ev(), ev()
            torch.cuda.synchronize()
            t0.record(stream)
            g.gf2_sigma_tau(h, G_tau, Sig, pc)
            t1.record(stream)
            torch.cuda.synchronize()
            Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
            sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
            g.gf2_fft_tau_to_iw(h, Sig, Sig_iw, sig12)
            Gi, Pi = torch.empty_like(G_iw), torch.empty_like(P)
            mu, _ = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, Gi, Pi)
            e1, e2 = g.gf2_energy(h, hc, F0, Pi, S, Gi, Sig_iw, sig12)
            E = s.e_nuc + e1 + e2
            row[name] = {"sigma_s_per_iter": t0.elapsed_time(t1) * 1e-3, "E": E}
            if ref is None:
                ref = (E, Pi)
            else:
                row[name]["abs_dE"] = abs(E - ref[0])
                row[name]["max_abs_dP"] = (Pi - ref[1]).abs().max().item()
        ctx.close()
        rows.append(row)
    worst = max(r_[p]["abs_dE"] for r_ in rows for p in ("bf16x3", "fp16x3", "bf16x6"))
    line = {"metric": "H32 STO-3G lattice (N=32): first-iteration |ΔE| of split Σ vs FP64 GPU Σ, per spacing",
            "value": rows[1]["fp64"]["sigma_s_per_iter"] / rows[1]["bf16x3"]["sigma_s_per_iter"],
            "unit": "x (FP64 Σ time / BF16x3 Σ time at 2.0 bohr)", "n_gpus": world, "steps": 1,
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3", "data": "synthetic (closed-form s-Gaussian integrals, RHF start)",
            "config": {"workload": "H32 2x4x4 STO-3G at 1.4/2.0/3.0 bohr, beta=100, n_tau=4097, n_iw=8192"},
            "worst_abs_dE": worst, "spacings": rows}
    if rank == 0:
        print(json.dumps(line))


def first_step_gpu(g, h, s, r, N, n_tau, n_iw, beta, prec, mu_hf=None):
    """The benchmark's step on an open context: finite-temperature HF state,
    G(i w) -> G(tau), Eq. Sigma, Sigma -> Sigma(i w), mu search at F_HF, energy.
    Returns (E, P, mu_hf, G_tau)."""
    import torch
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    S, hc, F0 = f64(s.S), f64(s.h), f64(r.F)
    G0 = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
    P0 = torch.zeros(N, N, dtype=torch.float64, device="cuda")
    if mu_hf is None:
        mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G0, P0)
    mom = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
    G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    g.gf2_tail_moments(h, S, F0, mu_hf, None, mom)
    g.gf2_fft_iw_to_tau(h, G0, mom, G_tau)
    Sig = torch.empty_like(G_tau)
    g.gf2_sigma_tau(h, G_tau, Sig, prec)
    Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
    sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
    g.gf2_fft_tau_to_iw(h, Sig, Sig_iw, sig12)
    del Sig
    P = torch.empty_like(P0)
    g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, G0, P)
    e1, e2 = g.gf2_energy(h, hc, F0, P, S, G0, Sig_iw, sig12)
    return s.e_nuc + e1 + e2, P, mu_hf, G_tau


def executed_share(N, eri):
    """Share of the 8 N^5 useful flops per time point that the split kernels
    execute: with the pair symmetry (im|qk) = (qk|im) of the integrals the
    sandwich (stages 1+2, half of the flops) computes only the unique stage-2
    tiles: 1056 of 2048 units per pair of time points at 64 wide, the 8256 of
    16384 units with i <= q at 128 wide."""
    pair_sym = bool(np.abs(eri - eri.transpose(2, 3, 0, 1)).max() <= 1e-12 * np.abs(eri).max())
    sym = (1056.0 / 2048.0 if N <= 64 else 8256.0 / 16384.0) if pair_sym else 1.0
    return (4.0 * sym + 4.0) / 8.0, pair_sym


def run_mesh(args, rank, world, dist):
    """The benchmark's system and step (H32 2x4x4 lattice, 6-31G, N = 64,
    beta = 100, n_iw = 8192; with --workload h64_mesh the H64 4x4x4 lattice,
    N = 128, beta = 200, n_iw = 16384) on the non-equidistant time grid the paper uses
    (Computational details): the uniform power mesh with --mesh P U (P halvings,
    U steps per interval: 2 (P+1) U + 1 points on a uniform grid of 2^(P+1) U
    intervals).  value = 8 N^5 n_points / step time; the energy and density are
    checked against the oracle's first step on the same mesh and on the 4097-point
    uniform grid (stored fixtures written from oracle/ only)."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    h64 = args.workload == "h64_mesh"
    if h64:  # H64 4x4x4 lattice, 6-31G (N = 128), beta = 200, 16384 frequencies
        s = gi.build_system("h64_lattice_631g")
        r = gi.rhf(s)
        n_iw, beta, tag = 16384, 200.0, "h64"
        label = "H64 lattice 4x4x4 at 2.0 bohr, 6-31G (N=128), beta=200"
    else:
        s, r = build_inputs()
        n_iw, beta, tag = WORKLOAD["n_iw"], WORKLOAD["beta"], "h32"
        label = "H32 lattice 2x4x4 at 2.0 bohr, 6-31G (N=64), beta=100"
    p_, u_ = args.mesh
    M, idx = g.power_mesh(p_, u_)
    N = s.nbf
    n_tau = len(idx)
    prec = PRECS[args.prec]
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    S, hcore, F0 = f64(s.S), f64(s.h), f64(r.F)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ctx = g.Context(N, None, n_iw, beta, grid=(M, idx))
    h = ctx.handle
    g.gf2_set_integrals(h, f64(s.eri))
    g.gf2_set_overlap(h, S)
    G_iw0 = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
    P0 = torch.zeros(N, N, dtype=torch.float64, device="cuda")
    mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G_iw0, P0)
    moments = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
    G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
    sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
    G_iw = torch.empty_like(G_iw0)
    P = torch.empty_like(P0)
    F_new = torch.empty_like(F0)

    def step(out, pc, sev=None):
        g.gf2_tail_moments(h, S, F0, mu_hf, None, moments)
        g.gf2_fft_iw_to_tau(h, G_iw0, moments, G_tau)
        if sev:
            sev[0].record(stream)
        g.gf2_sigma_tau(h, G_tau, Sig_tau, pc)
        if sev:
            sev[1].record(stream)
        g.gf2_fft_tau_to_iw(h, Sig_tau, Sig_iw, sig12)
        mu, nev = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, G_iw, P)
        g.gf2_fock(h, hcore, P, F_new)
        e1, e2 = g.gf2_energy(h, hcore, F0, P, S, G_iw, Sig_iw, sig12)
        out.append((s.e_nuc + e1 + e2, mu, nev))

    log = []
    for _ in range(args.warmup):
        step(log, prec)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    g.gf2_profile(h, False)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0, t1 = ev(), ev()
    sev = [(ev(), ev()) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.steps):
        step(log, prec, sev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms_step = max_over_ranks(t0.elapsed_time(t1) / args.steps, dist)
    sigma_ms = statistics.mean(a.elapsed_time(b) for a, b in sev)
    E_split, P_split = log[-1][0], P.clone()
    g.gf2_profile(h, True)
    for _ in range(args.steps):
        step(log, prec)
    torch.cuda.synchronize()
    prof, launches = g.gf2_profile_report(h)
    g.gf2_profile(h, False)
    # the same step with the FP64 GPU Sigma (and the other split precision)
    checks = {}
    for name in ["fp64"] + [x for x in ("fp16x3", "bf16x6") if x != args.prec]:
        step(log, PRECS[name])
        checks[name] = (log[-1][0], P.clone())
    checks[args.prec] = (E_split, P_split)
    fixtures = {}
    for key, path in (("same_mesh", f"{tag}_631g_first_step_pm{p_}x{u_}_w{n_iw}.json"),
                      ("uniform_4097", f"{tag}_631g_first_step_t4097_w{n_iw}.json")):
        fp = os.path.join(ROOT, "tests", "golden", path)
        if os.path.exists(fp):
            d = json.load(open(fp))
            P_or = torch.as_tensor(np.array(d["P"]), device="cuda")
            fixtures[key] = {"fixture": os.path.relpath(fp, ROOT), "E_oracle": d["E"],
                             **{name: {"abs_dE": abs(E - d["E"]), "max_abs_dP": (Pn - P_or).abs().max().item()}
                                for name, (E, Pn) in checks.items()}}
    useful = 8.0 * N ** 5 * n_tau
    _, _, bf16_sust, _ = measured_peaks()
    exec_frac, _ = executed_share(N, s.eri)
    line = {"metric": f"GF2 iteration on the non-equidistant time grid ({tag.upper()} 6-31G)",
            "value": useful / (ms_step * 1e-3) / 1e12 * world, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic (closed-form s-Gaussian integrals, RHF start)",
            "config": {"workload": (f"{label}, n_iw={n_iw}, "
                                    f"power mesh p={p_} u={u_}: {n_tau} time points on a {M}-interval grid"),
                       "step": "one GF2 outer iteration, all hot-path rows",
                       "parallelism": f"replicas x{world}"},
            "sigma": {"s_per_iter": sigma_ms * 1e-3, "tflops_useful": useful / (sigma_ms * 1e-3) / 1e12,
                      "issued_frac_of_bf16_build": useful * exec_frac * ISSUED[args.prec] / (sigma_ms * 1e-3)
                      / 1e12 / bf16_sust},
            "oracle_check": fixtures,
            "kernels": {k: {"launches": c, "ms_per_step": ms / args.steps} for k, (c, ms) in prof.items()},
            "gpu_launches": launches, "clocks": clocks, "mu_evaluations_per_step": log[-1][2]}
    ctx.close()
    if rank == 0:
        print(json.dumps(line))


def run_h64(args, rank, world, dist):
    """H64 4x4x4 lattice at 2.0 bohr, 6-31G (N = 128), beta = 200, n_tau = 8193,
    n_iw = 16384: one GF2 step through every row with the 128-wide split Sigma
    (time points in chunks of 16, intermediates 2 x 16 GB).  Accuracy: split vs
    FP64 GPU Sigma on sampled points of the full grid, and the first-step
    energy and density of the split path against the FP64 GPU path on a
    reduced grid (129 time points, 256 frequencies; the FP64 Sigma of the full
    grid would take about 30 minutes).  The FP64 GPU path itself is checked
    against the oracle at N = 128 by the GPU tests."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    s = gi.build_system("h64_lattice_631g")
    r = gi.rhf(s)
    N, beta = s.nbf, 200.0
    n_tau, n_iw = args.n_tau or 8193, args.n_iw or 16384
    prec = PRECS[args.prec]
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    S, hcore, F0 = f64(s.S), f64(s.h), f64(r.F)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ctx = g.Context(N, n_tau, n_iw, beta)
    h = ctx.handle
    g.gf2_set_integrals(h, f64(s.eri))
    g.gf2_set_overlap(h, S)
    G_iw0 = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
    P0 = torch.zeros(N, N, dtype=torch.float64, device="cuda")
    mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G_iw0, P0)
    moments = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
    G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
    sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
    G_iw = torch.empty_like(G_iw0)
    P = torch.empty_like(P0)
    F_new = torch.empty_like(F0)

    def step(out, sev=None):
        g.gf2_tail_moments(h, S, F0, mu_hf, None, moments)
        g.gf2_fft_iw_to_tau(h, G_iw0, moments, G_tau)
        if sev:
            sev[0].record(stream)
        g.gf2_sigma_tau(h, G_tau, Sig_tau, prec)
        if sev:
            sev[1].record(stream)
        g.gf2_fft_tau_to_iw(h, Sig_tau, Sig_iw, sig12)
        mu, nev = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, G_iw, P)
        g.gf2_fock(h, hcore, P, F_new)
        e1, e2 = g.gf2_energy(h, hcore, F0, P, S, G_iw, Sig_iw, sig12)
        out.append((s.e_nuc + e1 + e2, mu, nev))

    log = []
    for _ in range(args.warmup):
        step(log)
    torch.cuda.synchronize()
    g.gf2_profile(h, True)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0, t1 = ev(), ev()
    sev = [(ev(), ev()) for _ in range(args.steps)]
    t0.record(stream)
    for k in range(args.steps):
        step(log, sev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof, launches = g.gf2_profile_report(h)
    g.gf2_profile(h, False)
    ms_step = max_over_ranks(t0.elapsed_time(t1) / args.steps, dist)
    sigma_ms = statistics.mean(a.elapsed_time(b) for a, b in sev)
    useful = 8.0 * N ** 5 * n_tau
    issued = ISSUED[args.prec]
    exec_frac, pair_sym = executed_share(N, s.eri)
    _, bf16_burst, bf16_sust, peak_kind = measured_peaks()
    # split vs FP64 GPU Sigma on sampled points of the full grid
    pts = [1, 2, n_tau // 4, n_tau // 2, n_tau - 3]
    o64 = torch.empty(1, N, N, dtype=torch.float64, device="cuda")
    osp = torch.empty_like(o64)
    worst, t64 = 0.0, []
    for k in pts:
        a, b = ev(), ev()
        a.record(stream)
        g.gf2_sigma_tau_points(h, G_tau, k, 1, o64, 0)
        b.record(stream)
        g.gf2_sigma_tau_points(h, G_tau, k, 1, osp, prec)
        torch.cuda.synchronize()
        t64.append(a.elapsed_time(b))
        rel = ((osp - o64).abs().max() / o64.abs().max()).item()
        worst = max(worst, rel)
    fp64_s_per_iter = statistics.median(t64) * 1e-3 * n_tau
    prof_ms = {k: {"launches": c, "ms_per_step": ms / args.steps} for k, (c, ms) in prof.items()}
    ctx.close()
    del G_iw0, G_iw, Sig_iw, Sig_tau
    torch.cuda.empty_cache()
    # the same step on a reduced grid: split and FP64 GPU Sigma
    reduced = {}
    with g.Context(N, 129, 256, beta) as c2:
        g.gf2_set_integrals(c2.handle, f64(s.eri))
        g.gf2_set_overlap(c2.handle, S)
        E64, P64, _, _ = first_step_gpu(g, c2.handle, s, r, N, 129, 256, beta, 0)
        for name in sorted({args.prec, "fp16x3", "bf16x6"}):
            Es, Ps, _, _ = first_step_gpu(g, c2.handle, s, r, N, 129, 256, beta, PRECS[name])
            reduced[name] = {"abs_dE_vs_fp64_gpu": abs(Es - E64), "max_abs_dP": (Ps - P64).abs().max().item()}
    line = {"metric": "Σ(τ) s/iter & TFLOP/s at N=128 (H64 lattice): split vs FP64 GPU path",
            "value": useful / (ms_step * 1e-3) / 1e12 * world, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic (closed-form s-Gaussian integrals, RHF start)",
            "config": {"workload": f"H64 lattice 4x4x4 at 2.0 bohr, 6-31G (N=128), beta=200, n_tau={n_tau}, n_iw={n_iw}",
                       "step": "one GF2 outer iteration, all hot-path rows",
                       "l2": "inputs larger than L2 (G(iw) 4.3 GB, intermediates 32 GB)",
                       "parallelism": f"replicas x{world}"},
            "sigma": {"s_per_iter": sigma_ms * 1e-3, "tflops_useful": useful / (sigma_ms * 1e-3) / 1e12,
                      "executed_share_of_8n5": exec_frac, "stage2_pair_symmetry": pair_sym,
                      "tflops_issued": useful * exec_frac * issued / (sigma_ms * 1e-3) / 1e12,
                      "issued_frac_of_bf16_sustained": useful * exec_frac * issued / (sigma_ms * 1e-3) / 1e12
                      / bf16_sust,
                      "useful_equiv_frac_of_bf16_sustained": useful * issued / (sigma_ms * 1e-3) / 1e12 / bf16_sust,
                      "peak_source": peak_label(peak_kind, f"sustained BF16 {bf16_sust} TFLOP/s")},
            "fp64_gpu_path": {"sigma_s_per_iter": fp64_s_per_iter, "sample": f"points {pts}"},
            "speedup_split_vs_fp64_sigma": fp64_s_per_iter / (sigma_ms * 1e-3),
            "kernels": prof_ms, "gpu_launches": launches, "clocks": clocks,
            "mu_evaluations_per_step": log[-1][2],
            "accuracy": {"split_vs_fp64_gpu_sigma_max_rel": worst, "sampled_points": pts,
                         "reduced_grid_first_step": {"grid": "n_tau=129, n_iw=256", **reduced}}}
    if rank == 0:
        print(json.dumps(line))


def run_sigma_only(args, rank, world, dist):
    """The Sigma(tau) build alone on seeded random inputs (a real symmetric
    G(tau) per point and 8-fold symmetric integrals) of --n-bf basis functions
    and --n-tau time points: the case the kernel profiles are taken on."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    N, n_tau = args.n_bf, args.n_tau or 33
    prec = PRECS[args.prec]
    G = torch.as_tensor(gi.random_symmetric_g(N, n_tau, seed=11) * 0.3, device="cuda")
    v_host = gi.random_eri(N, seed=12)
    exec_frac, _ = executed_share(N, v_host)
    v = torch.as_tensor(v_host, device="cuda")
    del v_host
    out = torch.empty_like(G)
    stream = torch.cuda.current_stream()
    with g.Context(N, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, v)
        for _ in range(args.warmup):
            g.gf2_sigma_tau(ctx.handle, G, out, prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            g.gf2_sigma_tau(ctx.handle, G, out, prec)
        b.record(stream)
        torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    useful = 8.0 * N ** 5 * n_tau
    _, _, bf16_sust, _ = measured_peaks()
    if rank == 0:
        print(json.dumps({"metric": f"Σ(τ) build only, N={N}, {n_tau} time points", "value": useful / (ms * 1e-3) / 1e12,
                          "unit": "TFLOP/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                          "dtype": args.prec, "data": "synthetic (seeded random G(tau) and integrals)",
                          "executed_share_of_8n5": exec_frac,
                          "issued_frac_of_bf16_sustained": useful * exec_frac * ISSUED[args.prec] / (ms * 1e-3) / 1e12
                          / bf16_sust,
                          "useful_equiv_frac_of_bf16_sustained": useful * ISSUED[args.prec] / (ms * 1e-3) / 1e12
                          / bf16_sust}))


def run_df(args, rank, world, dist):
    """One GF2 iteration of the benchmark's system (H32 2x4x4 lattice, 6-31G,
    N = 64, beta = 100, n_iw = 8192) on density-fitted integrals: six
    even-tempered s exponents per atom (m = 192 fitted directions), on the
    power mesh --mesh P U.  The step is run_mesh's, with Sigma(tau) taken in the
    factor order of the fitted integrals in FP64 (gf2_sigma_tau_df: C = B G,
    X = Gbar C, U = X W, Sigma = -sum_Q C U; 2 m N^4 + 6 m N^3 flops per time
    point) and, beside it, by the four-stage split path (--prec) on the same
    fitted integrals.  value = the factor-order flops of the Sigma build per
    step / step time."""
    import torch
    import gf2_inputs as gi
    from gf2_inputs import density_fitting as dfi
    import paper_1405_3273_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    s, r = build_inputs()
    B_host = dfi.build_df(s.coords, s.basis)
    m, N = B_host.shape[0], s.nbf
    Bf = B_host.reshape(m, N * N)
    fit_err = float(np.abs(Bf.T @ Bf - s.eri.reshape(N * N, N * N)).max())
    n_iw, beta = WORKLOAD["n_iw"], WORKLOAD["beta"]
    p_, u_ = args.mesh
    M, idx = g.power_mesh(p_, u_)
    n_tau = len(idx)
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    S, hcore, F0 = f64(s.S), f64(s.h), f64(r.F)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ctx = g.Context(N, None, n_iw, beta, grid=(M, idx))
    h = ctx.handle
    g.gf2_set_df_integrals(h, f64(B_host))
    g.gf2_set_overlap(h, S)
    G_iw0 = torch.zeros(n_iw, N, N, dtype=torch.complex128, device="cuda")
    P0 = torch.zeros(N, N, dtype=torch.float64, device="cuda")
    mu_hf = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    mu_hf, _ = g.gf2_mu_search(h, S, F0, None, None, s.n_elec, mu_hf, G_iw0, P0)
    moments = torch.empty(4, N, N, dtype=torch.float64, device="cuda")
    G_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_tau = torch.empty(n_tau, N, N, dtype=torch.float64, device="cuda")
    Sig_iw = torch.empty(n_iw, N, N, dtype=torch.complex128, device="cuda")
    sig12 = torch.empty(2, N, N, dtype=torch.float64, device="cuda")
    G_iw = torch.empty_like(G_iw0)
    P = torch.empty_like(P0)
    F_new = torch.empty_like(F0)

    def step(out, factor_order, sev=None):
        g.gf2_tail_moments(h, S, F0, mu_hf, None, moments)
        g.gf2_fft_iw_to_tau(h, G_iw0, moments, G_tau)
        if sev:
            sev[0].record(stream)
        if factor_order:
            g.gf2_sigma_tau_df(h, G_tau, 0, n_tau, Sig_tau, 0)
        else:
            g.gf2_sigma_tau(h, G_tau, Sig_tau, PRECS[args.prec])
        if sev:
            sev[1].record(stream)
        g.gf2_fft_tau_to_iw(h, Sig_tau, Sig_iw, sig12)
        mu, nev = g.gf2_mu_search(h, S, F0, Sig_iw, sig12, s.n_elec, mu_hf, G_iw, P)
        g.gf2_fock(h, hcore, P, F_new)
        e1, e2 = g.gf2_energy(h, hcore, F0, P, S, G_iw, Sig_iw, sig12)
        out.append((s.e_nuc + e1 + e2, P.clone()))

    res = {}
    clocks = None
    for factor_order in (True, False):
        log = []
        for _ in range(args.warmup):
            step(log, factor_order)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(torch.cuda.current_device())
        if factor_order:
            sampler.start()
        t0, t1 = ev(), ev()
        sev = [(ev(), ev()) for _ in range(args.steps)]
        t0.record(stream)
        for k in range(args.steps):
            step(log, factor_order, sev[k])
        t1.record(stream)
        torch.cuda.synchronize()
        if factor_order:
            clocks = sampler.stop()
        res[factor_order] = {"ms_step": max_over_ranks(t0.elapsed_time(t1) / args.steps, dist),
                             "sigma_ms": statistics.mean(a.elapsed_time(b) for a, b in sev),
                             "E": log[-1][0], "P": log[-1][1]}
    g.gf2_profile(h, True)
    step([], True)
    torch.cuda.synchronize()
    prof, launches = g.gf2_profile_report(h)
    g.gf2_profile(h, False)
    ctx.close()
    df_flops = (2.0 * m * N ** 4 + 6.0 * m * N ** 3) * n_tau
    fo, sp = res[True], res[False]
    fp64_peak = 1.25 * (clocks["sm_mhz"] / 2070.0 if clocks else 1.0)
    dgemm_ms = prof.get("dgemm_fp64", (0, 0.0))[1]
    line = {"metric": "GF2 iteration on density-fitted integrals (H32 6-31G, m=192), factor-order FP64 Σ",
            "value": df_flops / (fo["ms_step"] * 1e-3) / 1e12 * world, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fo["ms_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form s-Gaussian integrals and auxiliary integrals, RHF start)",
            "config": {"workload": (f"H32 lattice 2x4x4 at 2.0 bohr, 6-31G (N={N}), beta={beta}, n_iw={n_iw}, "
                                    f"power mesh p={p_} u={u_}: {n_tau} time points; auxiliary set: "
                                    f"s exponents 0.3 x 2.6^k, k=0..5, on every atom (m={m})"),
                       "step": "one GF2 outer iteration, all hot-path rows",
                       "parallelism": f"replicas x{world}"},
            "fit": {"m": m, "max_abs_v_error": fit_err},
            "sigma_factor_order_fp64": {"s_per_build": fo["sigma_ms"] * 1e-3,
                                        "tflops": df_flops / (fo["sigma_ms"] * 1e-3) / 1e12,
                                        "frac_of_fp64_peak": df_flops / (fo["sigma_ms"] * 1e-3) / 1e12 / fp64_peak,
                                        "fp64_peak_tflops": fp64_peak,
                                        "peak_source": "derived: 1.25 TFLOP/s FP64 nominal at 2070 MHz, "
                                                       "scaled to the sampled clock",
                                        "dgemm_ms_per_build": dgemm_ms},
            f"sigma_four_stage_{args.prec}": {"s_per_build": sp["sigma_ms"] * 1e-3, "ms_per_step": sp["ms_step"],
                                              "abs_dE_vs_factor_order_fp64": abs(sp["E"] - fo["E"]),
                                              "max_abs_dP_vs_factor_order_fp64":
                                                  (sp["P"] - fo["P"]).abs().max().item()},
            "E_factor_order_fp64": fo["E"],
            "kernels": {k: {"launches": c, "ms": ms} for k, (c, ms) in prof.items()},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))


def run_converge(args, rank, world, dist):
    """Self-consistent GF2 on the linear H10 chain (STO-3G, 1.8 bohr, beta = 100,
    n_tau = 2049, n_iw = 4096) until the energy changes by less than 1e-8 Eh between
    outer iterations (or --max-outer), once with the FP64 Sigma and once per split
    precision; the converged energies and densities of the split runs against the
    FP64 run, and the wall time of each run."""
    import torch
    import gf2_inputs as gi
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import driver

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    s = gi.build_system("h10_chain_sto3g")
    r = gi.rhf(s)
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    runs = {}
    for name in ("fp64", "fp16x3", "bf16x6", "bf16x3"):
        ds = driver.to_device(s, r.F, mu0)
        t = time.perf_counter()
        run = driver.run_gf2(ds, prec=PRECS[name], max_outer=args.max_outer, e_tol=1e-8)
        torch.cuda.synchronize()
        runs[name] = {"seconds": time.perf_counter() - t, "energies": [e[0] for e in run.energies],
                      "P": run.P.cpu().numpy(), "mu": run.mu}
        run.ctx.close()
    ref = runs["fp64"]
    out = {}
    for name, x in runs.items():
        out[name] = {"seconds": x["seconds"], "outer_iterations": len(x["energies"]) - 1,
                     "E_final": x["energies"][-1], "energies": x["energies"], "mu": x["mu"]}
        if name != "fp64":
            out[name]["abs_dE_final"] = abs(x["energies"][-1] - ref["energies"][-1])
            out[name]["max_abs_dP_final"] = float(np.abs(x["P"] - ref["P"]).max())
    line = {"metric": "converged GF2 energy, linear H10 STO-3G: split Σ vs FP64 GPU Σ",
            "value": out["fp16x3"]["abs_dE_final"], "unit": "Eh (|ΔE| FP16x3 vs FP64 at convergence)",
            "n_gpus": world, "higher_is_better": False, "vs_baseline": None, "dtype": "fp16x3",
            "data": "synthetic (closed-form s-Gaussian integrals, RHF start)",
            "config": {"workload": "H10 chain 1.8 bohr, STO-3G (N=10), beta=100, n_tau=2049, n_iw=4096",
                       "stop": "|E_k - E_(k-1)| < 1e-8 Eh or max_outer"},
            "runs": out}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    rank, world, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
    elif args.workload == "batch":
        run_batch(args, rank, world, dist)
    elif args.workload == "h32_sto3g":
        run_h32_sto3g(args, rank, world, dist)
    elif args.workload == "converge":
        run_converge(args, rank, world, dist)
    elif args.workload in ("h32_mesh", "h64_mesh"):
        run_mesh(args, rank, world, dist)
    elif args.workload == "h64":
        run_h64(args, rank, world, dist)
    elif args.workload == "sigma":
        run_sigma_only(args, rank, world, dist)
    elif args.workload == "h32_df":
        run_df(args, rank, world, dist)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
