#!/usr/bin/env python
"""Benchmark of the LNV hot path on 4096-atom Si (8x8x8 diamond cells).

One "step" is one conjugate-gradient step of the LNV minimisation: the
energy and gradient (truncated block products, traces, the gradient
combine), the exact cubic line search (more products and traces) and the
update of L.  The headline value is mixed-precision steps per second: the
configuration's mixed mode, split-TF32 block products on the tensor cores
with FP32 accumulation (per product the faster of those and the FP32 FMA
schedules, timed by the first steps), float32 storage, float64 traces and
CG.  Beside it: FP32-FMA-only mixed steps, the float64 path, the runs to
|dOmega|/N < 1e-6 Ha/atom with their time to solution, the dominant
product's tensor-core and FMA rooflines against measured peaks, the
end-to-end number through the public API with host buffers (the call the
device-timed value makes, with its copies; and the same call with the
float64 evaluation of the result), and the CPU oracle timed on a row
sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batch     # 48 independent systems, 4x4 and 13x13 blocks
  python bench.py --workload sizes     # ms/step against atoms, 512 ... 32768 by default (O(N))
  python bench.py --workload oracle    # the CPU oracle on this host's cores (no GPU)

With N > 1 (torchrun) every rank runs an independent replica of the
workload on its own GPU (the path has no exchange step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import batch_workload, config_seed, diamond_si_positions, md_trajectory, sk_blocks  # noqa: E402

N_CELLS = 8
SIGMA = 0.05
R_S = R_H = 6.6
R_L = 10.0
MU = -2.0
B = 4
METRIC = "LNV steps/s & bsGEMM GFLOP/s, 4096-atom Si, mixed vs FP64 @1e-6 Ha/atom"
WORKLOAD = ("4096-atom Si (8x8x8 diamond cells, a=5.431 A, sigma=0.05 A, seed 2002077041), "
            "sp3 Slater-Koster H/S, 4x4 blocks, R_S=R_H=6.6 A, R_L=10 A, mu=-2 eV")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--fp64-steps", type=int, default=10)
    p.add_argument("--tol", type=float, default=1e-6,
                   help="|dOmega|/N (Ha/atom) at which the to-tolerance runs stop")
    p.add_argument("--no-tol", action="store_true", help="skip the runs to tolerance")
    p.add_argument("--cpu-sample-rows", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch-steps", type=int, default=3,
                   help="timed steps of the 48-system batched workload in the default line (0: skip)")
    p.add_argument("--md-steps", type=int, default=8,
                   help="extended-Lagrangian MD steps of the 4096-atom system (0: skip)")
    p.add_argument("--cells", default="4,6,8,10,12,16",
                   help="--workload sizes: diamond cells per edge of each system (8 n^3 atoms)")
    p.add_argument("--workload", default="si4096", choices=["si4096", "batch", "sizes", "oracle"],
                   help="si4096: the 4096-atom headline (default); batch: the 48-system batched "
                        "workload (24 systems with 4x4 blocks, 24 with 13x13); oracle: the CPU "
                        "oracle timed on the host cores (1 thread and all), no GPU")
    p.add_argument("--only-product", nargs="?", const="sl_qt", choices=["sl_qt", "ls_l", "xl", "tc_sl_qt"],
                   help="run only one kernel three times (for profilers): sl_qt, the roofline "
                        "product (default), ls_l, the bsgemm product, tc_sl_qt, the roofline product "
                        "on the tensor cores (LSQ_TF32X3), or xl, the XL-BOMD propagation of X with "
                        "dissipation (1728 atoms: 8 arrays of 210 MB)")
    p.add_argument("--product-cells", type=int, default=N_CELLS,
                   help="--only-product: diamond cells per edge of the system (8: the 4096-atom "
                        "workload; 6: 1728 atoms, a small case for multi-pass profiler captures)")
    return p.parse_args()


# ---- the CPU oracle on a row sample ------------------------------------------
def oracle_step_seconds(pos, cell, rows_per_step, seed):
    """Seconds of one oracle CG step (energy, gradient, cubic coefficients) at full size,
    estimated from a sample: every block product restricted to `rows_per_step` random
    rows (scaled by n / rows), all other work timed in full."""
    import oracle
    from oracle import lnv as OL
    m = OL.System(pos, cell)
    pH = m.pattern(R_H)
    H, S = sk_blocks(pos, cell, pH.rows(), pH.col)
    Hb, Sb = oracle.Bsr(pH, B, H), oracle.Bsr(pH, B, S)
    lnv = OL.Lnv(m, Sb, Hb, R_L, MU)
    L = OL.onsite_inverse_half(Sb, lnv.pat_L)
    n = pos.shape[0]
    rows = np.sort(np.random.default_rng(seed).choice(n, size=rows_per_step, replace=False))
    t0 = time.perf_counter()
    with OL.row_sample(rows) as smp:
        lnv.energy(L)
        G = lnv.gradient(L)
        G = 0.5 * (G + oracle.transpose(G, G.pat))
        D = -1.0 * G
        lnv.cubic(L, D, G)
    total = time.perf_counter() - t0
    mm = smp.mm_seconds
    return mm * n / rows_per_step + (total - mm), total


def host_cpu():
    """(cores, model name) of this host."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model", "hardware")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        # Arm hosts list an implementer and a part number instead of a model name
        try:
            ids = {}
            for ln in open("/proc/cpuinfo"):
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    ids.setdefault(k.strip().lower(), v.strip().lower())
            parts = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1",
                     "0xd49": "Neoverse-N2", "0xd8e": "Neoverse-N3", "0xd84": "Neoverse-V3"}
            if ids.get("cpu implementer") == "0x41" and ids.get("cpu part") in parts:
                model = "Arm " + parts[ids["cpu part"]]
        except OSError:
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count(), model


def run_reference(args):
    """The oracle on this host's cores, on the 4096-atom workload: each step is one oracle CG
    step (energy, gradient, cubic) whose block products are restricted to a random sample of
    rows and scaled by 4096 / rows (the products are row-separable), other work in full."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pos, cell = diamond_si_positions(N_CELLS, SIGMA, config_seed(1))
    import oracle
    oracle.build()
    oracle.build(openmp=True)
    threads = oracle.use_threads(0)
    ncpu, model = host_cpu()
    rows = max(16, args.cpu_sample_rows)
    for w in range(args.warmup):
        oracle_step_seconds(pos, cell, rows, 1000 + w)
    est, wall = [], 0.0
    for k in range(args.steps):
        e, t = oracle_step_seconds(pos, cell, rows, 2000 + k)
        est.append(e)
        wall += t
    sec = float(np.mean(est))
    v = 1.0 / sec
    sample = ("oracle CG step with each block product restricted to %d random rows of 4096 and "
              "scaled by 4096/%d (an extrapolation, not a timed full step), other work in full; "
              "%d steps, %.1f s of wall time in all" % (rows, rows, args.steps, wall))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "float64 oracle (CPU)"},
            "extrapolated": {"rows_sampled": rows, "scale": 4096.0 / rows, "wall_s": wall,
                             "note": "ms_per_step is the projected time of a full-size step, not "
                                     "a measured one"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": threads, "kind": "oracle",
                             "cpu_model": model, "host_cpus": ncpu, "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measured_peaks():
    """The machine's measured HBM copy bandwidth (GB/s), or the recipe's fallback figure."""
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of one float across all ranks (the timing rule: max over ranks)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps_per_rank, world, ms_per_step_max):
    """Whole-job steps/s: every rank runs its own replica, timed by the slowest rank."""
    return world * steps_per_rank / (steps_per_rank * ms_per_step_max / 1000.0)


# ---- clocks during the timed region -----------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "lsq_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        """Starts sampling every 50 ms and returns once the first sample is written (nvidia-smi
        takes a moment to start), so that the timed region that follows is covered."""
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.01)
        self.t_begin = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)  # one more sample after the timed region
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        # the first line was written before the timed region began
        for ln in lines[1:] if len(lines) > 1 else lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 50}


# ---- our arm -------------------------------------------------------------------
ROOFLINE_PRODUCT = "sl_qt_upper_rl"


def roofline_product(lsq, geom, SL, Q, out, precision=None):
    """The step's dominant product kernel: SL.Q^T on the upper triangle of L's range (the
    gradient terms and the line search's Z are products of this shape, three per step)."""
    return lsq.block_matmul(geom, B, SL, 3, Q, 5, out, 2, precision=lsq.F32 if precision is None else precision,
                            trans_b=True, triangle=2)


def traffic_of(fname, src, product_id):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a product kernel
    from a committed ncu summary under profiles/, or None when the summary is of another product
    or the kernel's source has changed since the capture (sha256 recorded in the summary)."""
    try:
        import hashlib
        tj = json.load(open(os.path.join(ROOT, "profiles", fname)))
        code = open(os.path.join(ROOT, "paper_2002_07704_gb300", "csrc", src), "rb").read()
        if tj.get("product_id") == product_id and tj.get(src.replace(".", "_") + "_sha256") == \
                hashlib.sha256(code).hexdigest():
            return tj.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def tensor_peaks():
    """(bf16, tf32) dense tensor TFLOP/s: the pool's measured cuBLAS bf16 burst, and tf32 at the
    nominal tf32/bf16 ratio of GB300's dense tensor rates (1.1 / 2.25 PFLOP/s)."""
    try:
        bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        bf16 = 1900.0
    return bf16, bf16 * 1.1 / 2.25
def xl_md_section(lsq, torch, stream, n_md, tol=1e-6):
    """Extended-Lagrangian MD steps of the headline system (Sec. 3.3) along a prescribed
    trajectory: per MD step the geometry (adopting the previous geometry's product
    schedules), H and S, S^-1 (Hotelling on R_L), the propagated X moved to the new patterns,
    L_0 = sym(X S^-1), and mixed-precision CG to tol.  Reports the CG iterations from that
    start against the previous step's L (moved to the new patterns) and the on-site start, the
    device time of the XL work (propagation, the moves of the history, the initial L), the
    wall time of each MD step (all three CG runs included, the model's H and S excluded), and
    the last step's S^-1 and CG on a fresh geometry with adopted schedules against its own
    tuning run."""
    K = 5
    kappa, alpha, c = lsq.XL_DISSIPATION_K5
    pos0, cell = diamond_si_positions(N_CELLS, SIGMA, config_seed(1))
    traj = md_trajectory(pos0, cell, n_md, seed=config_seed(1) + 77)
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    f64 = torch.float64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = {"xl": [], "previous_L": [], "onsite": []}
    xl_ms, prop_ms, move_ms, init_ms = [], [], [], []
    prev = None
    wall = []
    xl_start = None
    for n in range(n_md + 1):
        t_step = time.perf_counter()
        g = lsq.Geometry(torch.from_numpy(traj[n]).cuda(), cell, ranges)
        if prev is not None:
            g.adopt_schedules(prev[0])          # same ranges: no tuning run for this geometry
        rS, rL, rLS = g.range_id(R_S), g.range_id(R_L), g.range_id(R_L + R_S)
        rp, col = g.pattern(1)
        rp, col = rp.cpu().numpy(), col.cpu().numpy()
        t_hs = time.perf_counter()
        H, S = sk_blocks(traj[n], cell, np.repeat(np.arange(g.n_atoms), np.diff(rp)), col)
        t_hs = time.perf_counter() - t_hs          # the model's H and S: input, not timed
        Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
        ctx = lsq.Lnv(g, B, R_S, R_H, R_L)
        Xi = torch.zeros((g.nnzb(rL), B, B), dtype=f64, device="cuda")
        lsq.hotelling_inverse(g, B, Sd, rS, Xi, rL, rLS, 12, precision=lsq.F32)
        lsq.hotelling_inverse(g, B, Sd, rS, Xi, rL, rLS, 2, precision=lsq.F64, start=False)
        L = torch.zeros((g.nnzb(rL), B, B), dtype=f64, device="cuda")
        if n == 0:
            ctx.init_L(Sd, L)
            ctx.minimise(L, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=tol, precision=lsq.F32)
        else:
            gp, ctxp, hist, LSp, Lp_prev = prev
            rLSp = gp.range_id(R_L + R_S)
            lsq.xl_initial_L(g, B, rLS, torch.zeros((g.nnzb(rLS), B, B), dtype=f64, device="cuda"),
                             rL, Xi, rL, L, precision=lsq.F32)      # builds this geometry's plan
            torch.cuda.synchronize()
            Xn = torch.empty_like(hist[0])
            moved = [torch.empty((g.nnzb(rLS), B, B), dtype=f64, device="cuda") for _ in range(K + 1)]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            lsq.xl_propagate(gp, B, rLSp, hist, LSp, Xn, kappa, alpha, c)
            ev[1].record(stream)
            for src, dst in zip([Xn] + hist[:K], moved):
                lsq.pattern_remap(gp, rLSp, g, rLS, B, src, dst)
            ev[2].record(stream)
            lsq.xl_initial_L(g, B, rLS, moved[0], rL, Xi, rL, L, precision=lsq.F32)
            ev[3].record(stream)
            torch.cuda.synchronize()
            prop_ms.append(ev[0].elapsed_time(ev[1]))
            move_ms.append(ev[1].elapsed_time(ev[2]))
            init_ms.append(ev[2].elapsed_time(ev[3]))
            xl_ms.append(ev[0].elapsed_time(ev[3]))
            hist = moved
            Lprev = torch.zeros_like(L)
            lsq.pattern_remap(gp, gp.range_id(R_L), g, rL, B, Lp_prev, Lprev)
            Lon = torch.zeros_like(L)
            ctx.init_L(Sd, Lon)
            xl_start = L.clone()
            for name, Ls in (("previous_L", Lprev), ("onsite", Lon), ("xl", L)):
                rep = ctx.minimise(Ls, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=tol, precision=lsq.F32)
                its[name].append(int(rep["iterations"]))
            ctxp.close()
            gp.close()
        LS = torch.zeros((g.nnzb(rLS), B, B), dtype=f64, device="cuda")
        lsq.block_matmul(g, B, L, rL, Sd, rS, LS, rLS)
        if n == 0:
            hist = [LS.clone() for _ in range(K + 1)]
        prev = (g, ctx, hist, LS, L)
        torch.cuda.synchronize()
        wall.append(time.perf_counter() - t_step - t_hs)
    # the last MD step's S^-1 and XL-started CG on a fresh geometry of the same positions, with
    # the schedules adopted from the previous geometry and with its own tuning run
    ab = {}
    for adopt in (True, False):
        g2 = lsq.Geometry(torch.from_numpy(traj[n_md]).cuda(), cell, ranges)
        if adopt:
            g2.adopt_schedules(prev[0])
        ctx2 = lsq.Lnv(g2, B, R_S, R_H, R_L)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xi2 = torch.zeros((g2.nnzb(g2.range_id(R_L)), B, B), dtype=f64, device="cuda")
        rs2, rl2, rls2 = g2.range_id(R_S), g2.range_id(R_L), g2.range_id(R_L + R_S)
        lsq.hotelling_inverse(g2, B, Sd, rs2, Xi2, rl2, rls2, 12, precision=lsq.F32)
        lsq.hotelling_inverse(g2, B, Sd, rs2, Xi2, rl2, rls2, 2, precision=lsq.F64, start=False)
        L2 = xl_start.clone() if xl_start is not None else torch.zeros_like(prev[4])
        ctx2.minimise(L2, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=tol, precision=lsq.F32)
        torch.cuda.synchronize()
        ab["adopted_schedules_s" if adopt else "own_tuning_s"] = time.perf_counter() - t0
        ctx2.close()
        g2.close()
    m_ls = prev[0].nnzb(prev[0].range_id(R_L + R_S)) * B * B
    prev[1].close()
    prev[0].close()
    mean = lambda v: float(np.mean(v)) if v else None
    hbm_peak, hbm_kind = measured_peaks()
    # algorithmic bytes: the propagation reads K + 1 history arrays and L S and writes X(t + dt);
    # each move reads and writes one array of L S's range (float64)
    prop_bytes = (K + 3) * m_ls * 8
    move_bytes = (K + 1) * 2 * m_ls * 8
    bw = lambda nbytes, ms: nbytes / (ms * 1e-3) / 1e9 if ms else None
    return {"md_steps": n_md, "tol_ha_per_atom": tol, "cg_iterations_to_tol": its,
            "xl_ms_per_md_step": mean(xl_ms), "propagate_ms": mean(prop_ms),
            "move_history_ms": mean(move_ms), "initial_L_ms": mean(init_ms),
            "propagate_gbs": bw(prop_bytes, mean(prop_ms)), "move_history_gbs": bw(move_bytes, mean(move_ms)),
            "md_step_wall_s": wall,
            "last_step_sinv_and_cg_s": ab,
            "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": hbm_kind,
            "dissipation": {"K": K, "kappa": kappa, "alpha": alpha, "c": list(c)},
            "workload": ("4096-atom Si moving along a prescribed seeded trajectory (0.05 A "
                         "oscillations, periods 20-40 steps, ~0.01 A per step); X on R_L + R_S, "
                         "S^-1 from 12 float32 + 2 float64 Hotelling steps on R_L; L_0 = sym(X S^-1) with float32 "
                         "products; mixed CG")}


def run_ours(args):
    import torch
    import paper_2002_07704_gb300 as lsq

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lsq.build()
    lsq.load()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # --- measured FMA rates of this GPU (roofline denominators of the FMA kernels) ---
    ffma = lsq.measure_peak(lsq.F32)
    dfma = lsq.measure_peak(lsq.F64)

    # --- workload (one replica per rank) ---
    ncells = args.product_cells if args.only_product else N_CELLS
    pos, cell = diamond_si_positions(ncells, SIGMA, config_seed(1) + 1000 * rank)
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    geom = lsq.Geometry(torch.from_numpy(pos).cuda(), cell, ranges)
    rp, col = geom.pattern(1)
    rp, col = rp.cpu().numpy(), col.cpu().numpy()
    rows = np.repeat(np.arange(geom.n_atoms), np.diff(rp))
    H, S = sk_blocks(pos, cell, rows, col)
    Hd = torch.from_numpy(H).cuda()
    Sd = torch.from_numpy(S).cuda()
    ctx = lsq.Lnv(geom, B, R_S, R_H, R_L)
    L0 = torch.zeros((geom.nnzb(2), B, B), dtype=torch.float64, device="cuda")
    ctx.init_L(Sd, L0)

    if args.only_product:
        # one product three times (the first call tunes its plan)
        Lc, Sc = L0.float(), Sd.float()
        LS = torch.zeros((geom.nnzb(3), B, B), dtype=torch.float32, device="cuda")
        lsq.block_matmul(geom, B, Lc, 2, Sc, 0, LS, 3, precision=lsq.F32, trans_b=True)
        Qx = torch.randn((geom.nnzb(5), B, B), dtype=torch.float32, device="cuda",
                         generator=torch.Generator(device="cuda").manual_seed(5))
        Gx = torch.zeros((geom.nnzb(2), B, B), dtype=torch.float32, device="cuda")
        if args.only_product == "ls_l":
            LSL = torch.zeros((geom.nnzb(5), B, B), dtype=torch.float32, device="cuda")
            for _ in range(3):
                lsq.block_matmul(geom, B, LS, 3, Lc, 2, LSL, 5, precision=lsq.F32, trans_b=True)
        else:
            prec = lsq.TF32X3 if args.only_product == "tc_sl_qt" else lsq.F32
            for _ in range(3):
                roofline_product(lsq, geom, LS, Qx, Gx, precision=prec)
            if prec == lsq.TF32X3:
                geom.device_status()
                print("tensor-core plan:", json.dumps(geom.product_plan_info(3, 5, 2, 2)))
        torch.cuda.synchronize()
        print("only-product done: %d atoms" % geom.n_atoms)
        return

    def steps(L, k, prec):
        return ctx.minimise(L, Sd, Hd, MU, max_iter=k, precision=prec, refine_iter=0,
                            final_eval=False)

    # --- mixed precision (the configuration's mode: split-TF32 tensor-core products with FP32
    # accumulation, float64 traces and CG; per product the faster of those and the FP32 FMA
    # schedules, timed by the first steps): warm-up, then the timed steps ---
    L = L0.clone()
    steps(L, max(args.warmup, 2), lsq.TF32X3)
    L = L0.clone()
    clk = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    n0 = lsq.launch_count()
    clk.start()
    # a profiler started with --profile-from-start off sees exactly the timed steps
    torch.cuda.profiler.start()
    e0.record(stream)
    rep = steps(L, args.steps, lsq.TF32X3)
    e1.record(stream)
    torch.cuda.profiler.stop()
    barrier()
    clocks = clk.stop()
    launches = lsq.launch_count() - n0
    done = int(rep["iterations"])
    if done != args.steps:
        print("warning: the timed minimisation stopped after %d of %d steps (status %d)"
              % (done, args.steps, rep["status"]), file=sys.stderr)
    ms = e0.elapsed_time(e1) / max(done, 1)
    ms_all = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(done, world, ms_all)

    # --- float64 path, same steps from the same start ---
    L64 = L0.clone()
    steps(L64, 1, lsq.F64)
    L64 = L0.clone()
    barrier()
    e0.record(stream)
    rep64 = steps(L64, args.fp64_steps, lsq.F64)
    e1.record(stream)
    barrier()
    ms64 = e0.elapsed_time(e1) / max(int(rep64["iterations"]), 1)
    # accuracy of the mixed path: float64 Omega of both iterates after the same number of steps
    Lm = L0.clone()
    steps(Lm, args.fp64_steps, lsq.TF32X3)
    om_m, _ = ctx.energy_gradient(Lm, Sd, Hd, MU)
    om_d, _ = ctx.energy_gradient(L64, Sd, Hd, MU)
    acc = abs(om_m - om_d) / lsq.HARTREE_EV / geom.n_atoms

    # --- mixed precision with FP32 FMA products only (LSQ_F32) ---
    Lt = L0.clone()
    steps(Lt, args.warmup, lsq.F32)
    Lt = L0.clone()
    barrier()
    e0.record(stream)
    rep_f32 = steps(Lt, args.steps, lsq.F32)
    e1.record(stream)
    barrier()
    ms_f32 = e0.elapsed_time(e1) / max(int(rep_f32["iterations"]), 1)
    # the step's products (range ids: 0 R_S = R_H, 2 R_L, 3 R_L + R_S, 5 R_H + R_L + R_S) and the
    # kernel the timing chose for each
    STEP_PRODUCTS = [("L.S", 2, 0, 3, 0), ("SL.(Q+Q^T)^T lower", 3, 5, 2, 3), ("SL.Q^T upper", 3, 5, 2, 2),
                     ("P = D.S", 2, 0, 3, 0), ("QD = H'.P", 0, 3, 5, 0), ("F = P.D", 3, 2, 5, 1),
                     ("Z = P^T.QD^T", 3, 5, 2, 1)]
    choices, fixed = {}, []
    for name, ra_, rb_, rc_, tri in STEP_PRODUCTS:
        try:
            info = geom.product_plan_info(ra_, rb_, rc_, tri)
            choices[name] = {-1: "untimed", 0: "fp32 fma", 1: "tensor cores"}[info["auto_choice"]]
            if info["auto_choice"] >= 0:
                # the same choice as a fixed setting, for profiler runs of this bench
                fixed.append("%d:%d:%d:%d=%d" % (ra_, rb_, rc_, (0, 1, 1, 2)[tri], info["auto_choice"]))
        except lsq.LsqError:
            choices[name] = "fp32 fma (no tensor-core plan)"

    # --- to the tolerance of the metric: CG until |dOmega|/N < tol, the mixed paths followed by
    # their float64 refinement steps and a float64 final Omega; time to solution included ---
    to_tol = None
    if not args.no_tol:
        to_tol = {"tol_ha_per_atom": args.tol}
        for name, prec in (("fp64", lsq.F64), ("mixed_f32", lsq.F32), ("mixed_tf32x3", lsq.TF32X3)):
            # warm-up: every plan and schedule this run touches (the float64 refinement and the
            # final float64 evaluation included) is built and tuned before the timed call
            Lr = L0.clone()
            ctx.minimise(Lr, Sd, Hd, MU, max_iter=2, precision=prec, refine_iter=1, final_eval=True)
            Lr = L0.clone()
            barrier()
            e0.record(stream)
            r = ctx.minimise(Lr, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=args.tol, precision=prec,
                             refine_iter=2, final_eval=True)
            e1.record(stream)
            barrier()
            to_tol[name] = {"iterations": int(r["iterations"]), "iterations_fp64": int(r["iterations_fp64"]),
                            "status": int(r["status"]), "omega_ev": r["omega_ev"],
                            "omega_ha_per_atom": r["omega_ha_per_atom"], "ne": r["ne"],
                            "seconds": e0.elapsed_time(e1) / 1e3}
        for name in ("mixed_f32", "mixed_tf32x3"):
            to_tol[name]["vs_fp64_ha_per_atom"] = abs(to_tol[name]["omega_ev"] - to_tol["fp64"]["omega_ev"]) \
                / lsq.HARTREE_EV / geom.n_atoms

    # --- dominant kernel: LS.L (row form) timed alone on the same stream ---
    dt = torch.float32
    Lc = L.to(dt)
    Sc = Sd.to(dt)
    LS = torch.zeros((geom.nnzb(3), B, B), dtype=dt, device="cuda")
    LSL = torch.zeros((geom.nnzb(5), B, B), dtype=dt, device="cuda")
    lsq.block_matmul(geom, B, Lc, 2, Sc, 0, LS, 3, precision=lsq.F32, trans_b=True)
    trip = lsq.block_matmul(geom, B, LS, 3, Lc, 2, LSL, 5, precision=lsq.F32, trans_b=True)
    reps = 5
    barrier()
    e0.record(stream)
    for _ in range(reps):
        lsq.block_matmul(geom, B, LS, 3, Lc, 2, LSL, 5, precision=lsq.F32, trans_b=True)
    e1.record(stream)
    barrier()
    kms = e0.elapsed_time(e1) / reps
    flops = 2.0 * B ** 3 * trip
    hbm_peak, hbm_kind = measured_peaks()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    fp32_nominal = 152 * 128 * 2 * sm_max * 1e6 / 1e12   # FP32 FMA lanes x 2 flop x clock
    fp32_peak = ffma                                       # measured (lsq_measure_peak)

    # --- the step's dominant kernel, on the plan the step tuned ---
    Gx = torch.zeros((geom.nnzb(2), B, B), dtype=dt, device="cuda")
    rtrip = roofline_product(lsq, geom, LS, LSL, Gx)
    barrier()
    e0.record(stream)
    for _ in range(reps):
        roofline_product(lsq, geom, LS, LSL, Gx)
    e1.record(stream)
    barrier()
    rms = e0.elapsed_time(e1) / reps
    rflops = 2.0 * B ** 3 * rtrip
    # the same product on the tensor cores (LSQ_TF32X3), split conversions of both operands included
    roofline_product(lsq, geom, LS, LSL, Gx, precision=lsq.TF32X3)
    barrier()
    e0.record(stream)
    for _ in range(reps):
        roofline_product(lsq, geom, LS, LSL, Gx, precision=lsq.TF32X3)
    e1.record(stream)
    barrier()
    tms = e0.elapsed_time(e1) / reps
    geom.device_status()
    tinfo = geom.product_plan_info(3, 5, 2, 2)
    traffic_tc = traffic_of("traffic_tc.json", "tc.cu", "tc_" + ROOFLINE_PRODUCT)
    bf16_peak, tf32_peak = tensor_peaks()
    # the float64 path: algorithmic flops of one CG step (the step's products, Q formed afresh
    # every tenth step) over the measured DFMA rate
    step_trip = 0.0
    for name, ra_, rb_, rc_, tri in STEP_PRODUCTS + [("Q = H'.LS", 0, 3, 5, 0)]:
        Aa = torch.zeros((geom.nnzb(ra_), B, B), dtype=torch.float32, device="cuda")
        Bb = torch.zeros((geom.nnzb(rb_), B, B), dtype=torch.float32, device="cuda")
        Cc = torch.zeros((geom.nnzb(rc_), B, B), dtype=torch.float32, device="cuda")
        t_ = lsq.block_matmul(geom, B, Aa, ra_, Bb, rb_, Cc, rc_, precision=lsq.F32, trans_b=True,
                              triangle=tri)
        step_trip += t_ / 10.0 if name.startswith("Q =") else t_
        del Aa, Bb, Cc
    fp64_step_flops = 2.0 * B ** 3 * step_trip
    # algorithmic bytes: A and B read once, the upper half of C written (float32)
    abytes = (geom.nnzb(3) + geom.nnzb(5) + geom.nnzb(2) / 2.0) * B * B * 4
    traffic = traffic_of("traffic.json", "plan.cu", ROOFLINE_PRODUCT)

    # --- the sparse inverse overlap (Hotelling) on L's range, the LNV metric ---
    # float32 products from the scaled start, then float64 steps continuing from that X
    hot = {}
    Xh = torch.zeros((geom.nnzb(2), B, B), dtype=torch.float64, device="cuda")
    lsq.hotelling_inverse(geom, B, Sd, 0, Xh, 2, 3, 1, precision=lsq.F32)   # plans, warm-up
    lsq.hotelling_inverse(geom, B, Sd, 0, Xh, 2, 3, 1, precision=lsq.F64)
    for prec, k, name, start in ((lsq.F32, 10, "f32", True), (lsq.F64, 3, "f64", False)):
        barrier()
        e0.record(stream)
        dxs = lsq.hotelling_inverse(geom, B, Sd, 0, Xh, 2, 3, k, precision=prec, start=start)
        e1.record(stream)
        barrier()
        hot[name] = {"ms_per_iteration": e0.elapsed_time(e1) / k, "iterations": k,
                     "from": "scaled start" if start else "the float32 result",
                     "last_dx_fro": dxs[-1]}

    # --- steps to a tolerance: plain CG against CG in the metric X ~ S^-1 (X on S's range) ---
    tol = 1e-6
    mcg = {"tol_ha_per_atom": tol}
    Xs = torch.zeros((geom.nnzb(0), B, B), dtype=torch.float64, device="cuda")
    barrier()
    e0.record(stream)
    lsq.hotelling_inverse(geom, B, Sd, 0, Xs, 0, 3, 12, precision=lsq.F32)
    lsq.hotelling_inverse(geom, B, Sd, 0, Xs, 0, 3, 2, precision=lsq.F64, start=False)
    e1.record(stream)
    barrier()
    mcg["hotelling_ms"] = e0.elapsed_time(e1)
    for name, metric in (("plain", False), ("metric", True)):
        if metric:
            ctx.set_metric(Xs, 0, 3)
        Lt = L0.clone()
        barrier()
        e0.record(stream)
        rt = ctx.minimise(Lt, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=tol, precision=lsq.F32,
                          refine_iter=0, final_eval=False)
        e1.record(stream)
        barrier()
        mcg[name] = {"iterations": int(rt["iterations"]), "ms": e0.elapsed_time(e1),
                     "status": int(rt["status"])}
    # the same from the purified start (McWeeny purification of the grand-canonical start built
    # from H and X, 15 steps with float32 products), in the metric
    Lp = torch.zeros_like(L0)
    barrier()
    e0.record(stream)
    ctx.init_purify(Sd, Hd, MU, Xs, 0, 3, Lp, 15, precision=lsq.F32)
    e1.record(stream)
    barrier()
    mcg["purify_ms"] = e0.elapsed_time(e1)
    barrier()
    e0.record(stream)
    rt = ctx.minimise(Lp, Sd, Hd, MU, max_iter=300, tol_ha_per_atom=tol, precision=lsq.F32,
                      refine_iter=0, final_eval=False)
    e1.record(stream)
    barrier()
    mcg["metric_from_purified"] = {"iterations": int(rt["iterations"]), "ms": e0.elapsed_time(e1),
                                   "status": int(rt["status"])}
    ctx.set_metric(None, 0, 3)

    # --- canonical LNV: CG steps at fixed N_e (N0 from the grand-canonical iterate L) ---
    _, n0 = ctx.energy_gradient(L, Sd, Hd, MU)
    Lc = L.clone()
    ctx.minimise_canonical(Lc, Sd, Hd, n0, max_iter=2, precision=lsq.F32)   # warm-up
    Lc = L.clone()
    barrier()
    e0.record(stream)
    rc_, lam_ = ctx.minimise_canonical(Lc, Sd, Hd, n0, max_iter=args.steps, precision=lsq.F32)
    e1.record(stream)
    barrier()
    canon = {"steps_per_s": 1000.0 * int(rc_["iterations"]) / e0.elapsed_time(e1),
             "ms_per_step": e0.elapsed_time(e1) / max(int(rc_["iterations"]), 1),
             "steps": int(rc_["iterations"]), "n_electrons": n0,
             "ne_error_rel": abs(rc_["ne"] - n0) / n0, "lambda_ev": lam_,
             "workload": "mixed precision, N_e fixed at its value at the grand-canonical iterate"}

    # --- extended-Lagrangian MD steps (Sec. 3.3) ---
    xl = xl_md_section(lsq, torch, stream, args.md_steps) if args.md_steps > 0 else None

    # --- end to end through the public API, host buffers ---
    Lh = L0.cpu().pin_memory()
    Sh = Sd.cpu().pin_memory()
    Hh = Hd.cpu().pin_memory()
    Lout = torch.empty_like(Lh).pin_memory()

    def run_e2e(final_eval):
        barrier()
        t0 = time.perf_counter()
        Ldev = Lh.to("cuda", non_blocking=True)
        Sdev = Sh.to("cuda", non_blocking=True)
        Hdev = Hh.to("cuda", non_blocking=True)
        rep_ = ctx.minimise(Ldev, Sdev, Hdev, MU, max_iter=args.steps, precision=lsq.TF32X3,
                            refine_iter=0, final_eval=final_eval)
        Lout.copy_(Ldev, non_blocking=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, rep_

    # the same call the device-timed value makes, with the copies in and out and the report
    t_e2e, rep_e2e = run_e2e(False)
    e2e = {"value": world * args.steps / t_e2e, "unit": "steps/s",
           "h2d_bytes_per_step": int((Lh.numel() + Sh.numel() + Hh.numel()) * 8 / args.steps),
           "d2h_bytes_per_step": int(Lout.numel() * 8 / args.steps),
           "omega_ev": rep_e2e["omega_ev"],
           "definition": ("one lnv_minimise call of %d mixed steps from pinned host L, S, H (the call "
                          "the device-timed value makes), with the copy of L back and the report"
                          % args.steps)}
    # the same with the float64 evaluation of Omega and N_e at the result
    t_e2e64, rep_e2e64 = run_e2e(True)
    e2e_fp64_eval = {"value": world * args.steps / t_e2e64, "unit": "steps/s", "omega_ev": rep_e2e64["omega_ev"],
                     "definition": "as e2e, plus the float64 evaluation of Omega and N_e at the result"}

    # --- the 48-system batched workload (uneven sizes, 4x4 and 13x13 blocks), float32 products:
    # one grouped call over both halves against the halves run separately; single GPU only ---
    batch = None
    if world == 1 and args.batch_steps > 0:
        ctx.close()
        geom.close()
        del ctx, geom, L, L0, Lt, Lm, L64, Hd, Sd
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        batch = batch_section(lsq, torch, stream, args.batch_steps, 2, 0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        oracle.build(openmp=True)
        ncpu, model = host_cpu()
        oracle.use_threads(1)
        sec1, wall1 = oracle_step_seconds(pos, cell, args.cpu_sample_rows, 7)
        nthr = oracle.use_threads(0)
        rows_n = max(args.cpu_sample_rows, 4 * nthr)
        secn, walln = oracle_step_seconds(pos, cell, rows_n, 7)
        oracle.use_threads(1)
        cpu = {"value": 1.0 / secn, "unit": "steps/s", "cores": nthr, "kind": "oracle", "cpu_model": model,
               "host_cpus": ncpu,
               "sample": ("one oracle CG step (energy, gradient, cubic) with every block product "
                          "restricted to %d random rows of 4096 (on %d threads) and scaled by 4096/%d, "
                          "other work timed in full; %.1f s wall" % (rows_n, nthr, rows_n, walln)),
               "single_core": {"value": 1.0 / sec1, "cores": 1,
                               "sample": "the same with %d rows on 1 thread; %.1f s wall"
                                         % (args.cpu_sample_rows, wall1)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3",
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "precision": "mixed: split-TF32 (hi + lo) block products on the tensor cores with "
                                    "FP32 accumulation where the per-product timing picks them, FP32 FMA "
                                    "elsewhere; float32 storage, float64 traces and CG",
                       "l2": "inputs larger than L2 (LSL alone is 885 MB in float32)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "product_kernels": choices,
                       "product_choice_setting": "LSQ_TC_CHOICE=" + ",".join(sorted(set(fixed)))},
            "fp64": {"steps_per_s": 1000.0 / ms64, "ms_per_step": ms64, "steps": args.fp64_steps,
                     "roofline": {"bound": "fp64", "achieved": fp64_step_flops / ms64 / 1e9, "peak": dfma,
                                  "unit": "TFLOP/s", "frac": fp64_step_flops / ms64 / 1e9 / dfma,
                                  "flops_per_step": fp64_step_flops,
                                  "peak_note": "measured DFMA loop (lsq_measure_peak)"}},
            "mixed_f32": {"steps_per_s": 1000.0 / ms_f32, "ms_per_step": ms_f32,
                          "steps": int(rep_f32["iterations"]),
                          "precision": "FP32 FMA products only (LSQ_F32), float64 traces and CG"},
            "mixed_vs_fp64_omega_ha_per_atom": acc,
            "mixed_vs_fp64_same_steps": {"steps": args.fp64_steps, "ha_per_atom": acc},
            "mixed_vs_fp64_at_tol": to_tol,
            "bsgemm": {"product": "LS.L truncated to 23.2 A (P2 of the product schedule, every block)",
                       "triples": trip,
                       "gflops": flops / kms / 1e6, "ms": kms, "frac_fp32_peak": flops / kms / 1e9 / fp32_peak},
            "roofline": {"bound": "tensor", "kernel": "k_tc_product (LSQ_TF32X3)",
                         "product": "SL.Q^T on the upper triangle of the 10 A range (A 16.6 A, B 23.2 A): "
                                    "the shape of three of the step's products, which the mixed step runs "
                                    "on the tensor cores",
                         "triples": rtrip, "ms": tms,
                         "achieved": 512.0 * tinfo["dense_triples"] / tms / 1e9, "unit": "TFLOP/s",
                         "achieved_note": "tensor flops the MMAs execute per launch (4 x 128 per dense block "
                                          "triple: hi/lo x hi/lo, zero blocks of the tiles included) over the "
                                          "launch time, split conversions of both operands included",
                         "peak": tf32_peak, "frac": 512.0 * tinfo["dense_triples"] / tms / 1e9 / tf32_peak,
                         "peak_note": "dense tf32 of measured: cuBLAS bf16 burst (%.0f) x 1.1 / 2.25 (the "
                                      "nominal tf32 / bf16 ratio)" % bf16_peak,
                         "traffic": traffic_tc,
                         "algorithmic_tflops": rflops / tms / 1e9,
                         "useful_fraction": tinfo["triples"] / max(tinfo["dense_triples"], 1),
                         "gathered_gbs": 128.0 * tinfo["blocks_copied"] / tms / 1e6,
                         "gathered_bytes": 128 * tinfo["blocks_copied"],
                         "block_slots": tinfo["block_slots"],
                         "gathered_note": "128-byte split blocks copied from L2/HBM into shared memory per "
                                          "launch; the other block slots of the tiles are zeros stored in "
                                          "shared memory",
                         "bound_note": "gathering the operand blocks (scattered 128-byte lines through L2) "
                                       "bounds this kernel, not the tensor pipe",
                         "vs_fma": rms / tms},
            "roofline_fma": {"bound": "alu", "achieved": rflops / rms / 1e9, "peak": fp32_peak,
                             "unit": "TFLOP/s", "frac": rflops / rms / 1e9 / fp32_peak,
                             "traffic": traffic,
                             "product": "the same SL.Q^T with FP32 FMA (LSQ_F32)",
                             "triples": rtrip, "ms": rms,
                             "kernel": "k_mm_plan_b4_rb<float, ...> (schedule picked by the autotuner)",
                             "hbm_frac": abytes / rms / 1e6 / hbm_peak, "hbm_peak_kind": hbm_kind,
                             "peak_note": "measured FFMA loop (lsq_measure_peak); nominal below",
                             "peak_nominal": fp32_nominal, "frac_nominal": rflops / rms / 1e9 / fp32_nominal},
            "hotelling": dict(hot, workload="X = S^-1 approximated on the 10 A range by "
                                             "X <- 2X - (X S) X from X0 = S / s^2, the LNV metric of Sec. 2.3.2"),
            "canonical": canon,
            "xlbomd": xl,
            "metric_cg": dict(mcg, workload="mixed-precision CG from L0 until |dOmega|/N < tol; "
                                               "metric: X from 12 float32 + 2 float64 Hotelling steps "
                                               "on the 6.6 A range"),
            "clocks": clocks,
            "e2e": e2e,
            "e2e_with_fp64_eval": e2e_fp64_eval,
            "batch": batch,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "last_report": {"mixed": rep, "fp64": rep64, "mixed_f32": rep_f32, "e2e": rep_e2e,
                            "e2e_with_fp64_eval": rep_e2e64},
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ---- the batched workload ----------------------------------------------------------
BATCH_R_L = 8.0


def batch_section(lsq, torch, stream, steps, warmup, fp64_steps):
    """The 48-system batched workload (synth.batch_workload): the 4x4 half and the 13x13 half
    each one block-diagonal geometry and LNV context.  Timed: (1) one grouped call over both
    halves (lsq_lnv_minimise_batch_group: every product of a step one persistent launch over
    the 48 systems, steps replayed as one CUDA graph), float32 products; (2) each half alone
    with its tuned product kernels (lsq_lnv_minimise_batch), float32 and float64.  Host setup
    (positions, H and S on the host) is not timed."""
    W = batch_workload()
    ranges = lsq.lnv_required_ranges(R_S, R_H, BATCH_R_L)
    parts = {}
    t0 = time.perf_counter()
    for b in (4, 13):
        ids = [s for s in range(len(W)) if W[s]["b"] == b]
        geoms, Hs, Ss = [], [], []
        for s in ids:
            w = W[s]
            pos, cell = diamond_si_positions(w["n"], w["sigma"], w["seed"])
            g = lsq.Geometry(torch.from_numpy(pos).cuda(), cell, ranges)
            rp, col = g.pattern(1)
            rp, col = rp.cpu().numpy(), col.cpu().numpy()
            rows = np.repeat(np.arange(g.n_atoms), np.diff(rp))
            H, S = sk_blocks(pos, cell, rows, col, b=b, perturb_seed=w["perturb_seed"])
            geoms.append(g)
            Hs.append(H)
            Ss.append(S)
        bg = lsq.concat_geometries(geoms)
        for g in geoms:
            g.close()
        Hd = torch.from_numpy(np.concatenate(Hs)).cuda()
        Sd = torch.from_numpy(np.concatenate(Ss)).cuda()
        ctx = lsq.Lnv(bg, b, R_S, R_H, BATCH_R_L)
        L0 = torch.zeros((bg.nnzb(2), b, b), dtype=torch.float64, device="cuda")
        ctx.init_L(Sd, L0)
        parts[b] = {"ids": ids, "geom": bg, "ctx": ctx, "H": Hd, "S": Sd, "L0": L0,
                    "atoms": int(sum(8 * W[s]["n"] ** 3 for s in ids))}
    setup = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mus = {b: [MU] * len(parts[b]["ids"]) for b in parts}

    def timed(fn):
        torch.cuda.synchronize()
        n0 = lsq.launch_count()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1), lsq.launch_count() - n0

    # (1) grouped: both halves in one call per timing
    order = (4, 13)
    ctxs = [parts[b]["ctx"] for b in order]
    Ss = [parts[b]["S"] for b in order]
    Hs = [parts[b]["H"] for b in order]
    mu_l = [mus[b] for b in order]
    kw = dict(precision=lsq.F32, refine_iter=0, final_eval=False)
    lsq.minimise_batch_group(ctxs, [parts[b]["L0"].clone() for b in order], Ss, Hs, mu_l,
                             max_iter=max(warmup, 2), **kw)
    Ls = [parts[b]["L0"].clone() for b in order]
    reps, ms, nl = timed(lambda: lsq.minimise_batch_group(ctxs, Ls, Ss, Hs, mu_l, max_iter=steps, **kw))
    grouped = {"ms_per_step": ms / steps, "system_steps_per_s": len(W) * 1000.0 * steps / ms,
               "steps": steps, "host_launches": nl,
               "status": sorted(set(int(r["status"]) for rr in reps for r in rr)),
               "definition": "one lsq_lnv_minimise_batch_group call over both halves; per step one "
                             "CUDA graph, each product one persistent launch over all 48 systems "
                             "(the call's first step runs context by context and builds the graphs)"}
    # (2) each half alone, tuned kernels; float64 last (it grows the product buffers to 8 bytes)
    halves = {}
    for b in order:
        P = parts[b]
        out = {"systems": len(P["ids"]), "atoms": P["atoms"]}
        for prec, k, name in ((lsq.F32, steps, "mixed"), (lsq.F64, fp64_steps if b == 4 else min(fp64_steps, 1), "fp64")):
            if k <= 0:
                continue
            if name == "fp64" and b == 13 and 4 in parts:
                # the 4x4 half is done: free it before the 13x13 float64 buffers are grown
                for key in ("ctx", "geom"):
                    parts[4][key].close()
                del parts[4]
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            P["ctx"].minimise_batch(P["L0"].clone(), P["S"], P["H"], mus[b], max_iter=max(warmup, 2) if name == "mixed" else 1,
                                    precision=prec, refine_iter=0, final_eval=False)
            L = P["L0"].clone()
            reps_h, ms_h, nl_h = timed(lambda: P["ctx"].minimise_batch(L, P["S"], P["H"], mus[b], max_iter=k,
                                                                      precision=prec, refine_iter=0, final_eval=False))
            out[name] = {"ms_per_batch_step": ms_h / k, "system_steps_per_s": len(P["ids"]) * 1000.0 * k / ms_h,
                         "steps": k, "host_launches": nl_h, "status": sorted(set(int(r["status"]) for r in reps_h))}
        halves["b%d" % b] = out
    for P in parts.values():
        P["ctx"].close()
        P["geom"].close()
    parts.clear()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    back_to_back = halves["b4"]["mixed"]["ms_per_batch_step"] + halves["b13"]["mixed"]["ms_per_batch_step"]
    return {"grouped": grouped, "halves": halves, "setup_s": setup,
            "halves_back_to_back": {"ms_per_step": back_to_back, "system_steps_per_s": len(W) * 1000.0 / back_to_back}}


def run_batch(args):
    """48 uneven Si systems (synth.batch_workload), float32 products: headline = one grouped
    call over both halves (batch_section)."""
    import torch
    import paper_2002_07704_gb300 as lsq
    lsq.build()
    lsq.load()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    sec = batch_section(lsq, torch, stream, args.steps, args.warmup, args.fp64_steps)
    clocks = clk.stop()
    W = batch_workload()
    line = {
        "metric": "batched LNV system-steps/s, 48 uneven Si systems (64-2744 atoms; b=4 and b=13)",
        "value": sec["grouped"]["system_steps_per_s"], "unit": "system-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec["grouped"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "synth.batch_workload(): 48 diamond-Si systems, n^3 cells with n "
                               "uniform in 2..7, sigma uniform in 0.05..0.15 A, R_S=R_H=6.6 A, "
                               "R_L=8 A, mu=-2 eV; systems 0-23 4x4 blocks, 24-47 13x13",
                   "precision": "float32 products, float64 traces/CG",
                   "step": "one CG step of all 48 systems: one grouped call, each product one "
                           "persistent launch over both halves"},
        "batch": sec,
        "clocks": clocks,
    }
    print(json.dumps(line))


def run_sizes(args):
    """Mixed-precision step time against system size (the O(N) claim of Sec. 2.3.2): the
    si4096 workload's recipe at n x n x n diamond cells for each n of --cells, one line."""
    import torch
    import paper_2002_07704_gb300 as lsq
    torch.cuda.set_device(0)
    lsq.build()
    lsq.load()
    stream = torch.cuda.current_stream()
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    out = []
    for nc in [int(x) for x in args.cells.split(",")]:
        pos, cell = diamond_si_positions(nc, SIGMA, config_seed(1))
        free0, total = torch.cuda.mem_get_info()
        geom = lsq.Geometry(torch.from_numpy(pos).cuda(), cell, ranges)
        rp, col = geom.pattern(1)
        rp, col = rp.cpu().numpy(), col.cpu().numpy()
        rows = np.repeat(np.arange(geom.n_atoms), np.diff(rp))
        H, S = sk_blocks(pos, cell, rows, col)
        Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
        ctx = lsq.Lnv(geom, B, R_S, R_H, R_L)
        L0 = torch.zeros((geom.nnzb(2), B, B), dtype=torch.float64, device="cuda")
        ctx.init_L(Sd, L0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(prec):
            L = L0.clone()
            ctx.minimise(L, Sd, Hd, MU, max_iter=max(args.warmup, 2), precision=prec, refine_iter=0,
                         final_eval=False)
            L = L0.clone()
            torch.cuda.synchronize()
            e0.record(stream)
            rep = ctx.minimise(L, Sd, Hd, MU, max_iter=args.steps, precision=prec, refine_iter=0,
                               final_eval=False)
            e1.record(stream)
            torch.cuda.synchronize()
            done = max(int(rep["iterations"]), 1)
            return e0.elapsed_time(e1) / done, done

        ms, done = timed(lsq.F32)
        ms_tc, _ = timed(lsq.TF32X3)
        free1, _ = torch.cuda.mem_get_info()
        n = geom.n_atoms
        out.append({"atoms": n, "cells": nc, "steps": done, "ms_per_step": ms,
                    "us_per_atom_step": ms * 1e3 / n,
                    "tf32x3": {"ms_per_step": ms_tc, "us_per_atom_step": ms_tc * 1e3 / n},
                    "nnzb": {"S": geom.nnzb(0), "L": geom.nnzb(2), "LSL": geom.nnzb(5)},
                    "device_gb": (free0 - free1) / 1e9})
        print("sizes: %d atoms, F32 %.3f ms/step (%.3f us/atom-step), TF32X3 %.3f ms/step (%.3f), %.1f GB" %
              (n, ms, ms * 1e3 / n, ms_tc, ms_tc * 1e3 / n, (free0 - free1) / 1e9), file=sys.stderr)
        ctx.close()
        geom.close()
        del ctx, geom, L0, Hd, Sd
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "mixed-precision LNV ms/step against atoms (O(N)); ms_per_step is float32 FMA "
                                "products, tf32x3 the configuration's mode", "unit": "ms/step",
                      "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "Si diamond n x n x n cells, sigma 0.05 A, R_S=R_H=6.6 A, "
                                             "R_L=10 A, 4x4 blocks, mu=-2 eV"},
                      "sizes": out}))


def run_only_xl():
    """Three launches of lsq_xl_propagate (six history entries, the K = 5 dissipation) on L S's
    range of 1728-atom Si (6x6x6 cells), random arrays; for profilers."""
    import torch
    import paper_2002_07704_gb300 as lsq
    lsq.build()
    lsq.load()
    pos, cell = diamond_si_positions(6, SIGMA, config_seed(1))
    g = lsq.Geometry(torch.from_numpy(pos).cuda(), cell, lsq.lnv_required_ranges(R_S, R_H, R_L))
    r = g.range_id(R_L + R_S)
    gen = torch.Generator(device="cuda").manual_seed(3)
    A = [torch.randn((g.nnzb(r), B, B), dtype=torch.float64, device="cuda", generator=gen) for _ in range(8)]
    kappa, alpha, c = lsq.XL_DISSIPATION_K5
    for _ in range(3):
        lsq.xl_propagate(g, B, r, A[:6], A[6], A[7], kappa, alpha, c)
    torch.cuda.synchronize()
    print("only-product xl done: %d values per array" % A[0].numel())


def run_oracle(args):
    """The CPU oracle on this host's cores, single-threaded and on all cores (its OpenMP build):
    the 64-atom configuration in full (20 CG steps), the three single products of the 4096-atom
    configuration on sampled rows (scaled by 4096 / rows; inputs are random blocks on the
    products' patterns, the time does not depend on the values), and CG steps of the 512-atom
    sub-cell of the 32768-atom configuration.  No GPU is used."""
    import oracle
    from oracle import lnv as OL
    oracle.build()
    oracle.build(openmp=True)
    ncpu, model = host_cpu()
    out = {"metric": "oracle (CPU) timings", "cpu_model": model, "host_cpus": ncpu}

    def lnv_case(ncell, sigma, seed, R_L):
        pos, cell = diamond_si_positions(ncell, sigma, seed)
        m = OL.System(pos, cell)
        pH = m.pattern(R_H)
        H, S = sk_blocks(pos, cell, pH.rows(), pH.col)
        Hb, Sb = oracle.Bsr(pH, B, H), oracle.Bsr(pH, B, S)
        lnv = OL.Lnv(m, Sb, Hb, R_L, MU)
        return lnv, OL.onsite_inverse_half(Sb, lnv.pat_L)

    for threads in (1, 0):
        nthr = oracle.use_threads(threads)
        key = "threads_%d" % nthr
        res = {}
        lnv, L0 = lnv_case(2, SIGMA, config_seed(0), 8.0)
        t0 = time.perf_counter()
        OL.minimise(lnv, L0, 20)
        res["cfg0_64_atoms_20_cg_steps_s"] = time.perf_counter() - t0
        lnv, L0 = lnv_case(4, 0.1, config_seed(4), R_L)
        OL.minimise(lnv, L0, 1)
        t0 = time.perf_counter()
        OL.minimise(lnv, L0, 2)
        res["cfg4_512_atom_subcell_s_per_cg_step"] = (time.perf_counter() - t0) / 2
        pos, cell = diamond_si_positions(N_CELLS, SIGMA, config_seed(1))
        P = {R: oracle.neighbour_list(pos, cell, R) for R in (R_S, R_L, R_L + R_S, R_H + R_L + R_S)}
        rng = np.random.default_rng(11)
        rnd = lambda R: oracle.Bsr(P[R], B, rng.standard_normal((P[R].nnzb, B, B)))
        rows = np.sort(rng.choice(4096, size=max(64, 4 * nthr), replace=False))
        prods = {}
        for name, ra, rb, rc in (("L.S", R_L, R_S, R_L + R_S), ("LS.L", R_L + R_S, R_L, R_H + R_L + R_S),
                                 ("LSL.SL|R_H", R_H + R_L + R_S, R_L + R_S, R_H)):
            A_, B_ = rnd(ra), rnd(rb)
            t0 = time.perf_counter()
            _, trip = oracle.matmul(A_, B_, P[rc], rows=rows)
            dt = time.perf_counter() - t0
            prods[name] = {"rows": int(rows.size), "s_sampled": dt, "s_full_estimate": dt * 4096 / rows.size,
                           "gflops": 2.0 * B ** 3 * trip / dt / 1e9}
        res["cfg1_products"] = prods
        out[key] = res
        print(json.dumps({key: res}), file=sys.stderr, flush=True)
    oracle.use_threads(1)
    print(json.dumps(out))


def main():
    args = parse()
    if args.only_product == "xl":
        run_only_xl()
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "oracle":
        run_oracle(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "sizes":
        run_sizes(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
