"""Benchmark of the COLA particle-mesh hot path on GB300.

One bench step = one whole mock realisation of the 512^3-particle / 1024^3-mesh / 1024 Mpc/h
workload: 2LPT initial conditions from a new seed, 10 COLA steps (deposit, FFT Poisson solve
with gradient and CIC deconvolution, inverse FFTs, gather + kick + drift) and the 100-bin
power spectrum. The metric is particle-updates per second (N_p^3 x 10 per step / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

With --gpus N > 1 (launched by torchrun) every rank runs independent mocks (replicas, no
data-path collective); the time is the max over ranks. The reference arm times the FP64
CPU oracle on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1506_03737_gb300 import workloads  # noqa: E402

# Algorithmic bytes (minimum HBM traffic) per COLA step for this data layout:
# particles 96 B per particle-update; mesh 80 B per cell.
ALG_BYTES_PARTICLE = 96
ALG_BYTES_CELL = 80
# Per-kernel algorithmic bytes per cell (mesh kernels) or particle (particle kernels).
ALG_PHASE = {
    "poisson": ("cell", 12),     # z pass: read the half spectrum, write the two inverse-z bases
    "fft_inv": ("cell", 20),     # inverse y: read the 2 bases, write 3 spectra
    "fft_inv_x": ("cell", 24),   # inverse x: read 3 half spectra, write 3 real force meshes
    "fft_fwd": ("cell", 12),     # forward passes: read int64 density, write half spectrum
    "deposit": ("cell", 16),     # atomic read-modify-write of the int64 mesh (+16 B/particle below)
    "gather": ("particle", 80),  # read pos, mom, psi1, psi2, write pos, mom (+12 B/cell below)
}
EXTRA = {"deposit": ("particle", 16), "gather": ("cell", 12)}
# The phases of a COLA step (the reordering of the particles by cell included when it runs).
STEP_PHASES = ("sort", "deposit", "fft_fwd", "poisson", "fft_inv", "fft_inv_x", "gather")
# Single-kernel phases, and the DRAM bytes (read + write) ncu measured for each kernel at
# 256^3 particles / 512^3 mesh (per launch, MB), scaled to other sizes with N_m = 2 N_p by the
# cell count: force z pass 538.8 + 1017.2, inverse x 1610.7 + 1561.6, force y inverse
# 1073.9 + 1546.3, gather 2494.7 + 454.1, deposit 1243.8 + 792.8.
DRAM_512 = {"poisson": 1556.0e6, "fft_inv_x": 3172.3e6, "fft_inv": 2620.2e6, "gather": 2948.8e6,
            "deposit": 2036.6e6}
# Phases that run another kernel at 1024^3 than the one measured at 512^3 (the force z pass there
# is the paired-lane kernel): their DRAM bytes per launch measured at 1024^3 (4515.6 + 8688.3 MB).
DRAM_1024 = {"poisson": 13203.9e6}


def roofline(phase_ms, phase_n, np_, nm, hbm):
    """Roofline object of the dominant kernel: the single-kernel phase with the largest total time.
    achieved = its algorithmic bytes per call / its mean call time; traffic = the ncu DRAM bytes
    per call measured at 512^3, scaled by the cell count (None off the N_m = 2 N_p family), or
    measured at 1024^3 for a kernel that only runs there."""
    dom = max(DRAM_512, key=lambda k: phase_ms[k])
    units = {"cell": nm ** 3, "particle": np_ ** 3}
    unit, b = ALG_PHASE[dom]
    nbytes = b * units[unit]
    if dom in EXTRA:
        nbytes += EXTRA[dom][1] * units[EXTRA[dom][0]]
    per_call_ms = phase_ms[dom] / max(int(phase_n[dom]), 1)
    achieved = nbytes / (per_call_ms / 1e3) / 1e9
    if nm == 1024 and dom in DRAM_1024:
        traffic = DRAM_1024[dom]
    else:
        traffic = DRAM_512[dom] / 512 ** 3 * nm ** 3 if nm == 2 * np_ else None
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "alg_bytes": nbytes}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cola_512p_1024m_1024mpc")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-study", action="store_true")
    ap.add_argument("--sort", type=int, default=None,
                    help="reorder the particles by cell every K steps (profiling aid; the default is the library's)")
    ap.add_argument("--sort-tiles", type=int, default=None,
                    help="order of the reordering: tiles of 64 x T x T cells, T in 1, 2, 4, 8 (profiling aid)")
    ap.add_argument("--deposit-tiles", type=int, default=None,
                    help="deposit tiles of 64 x T x T cells, T in 0, 2, 4, 8 (profiling aid; the default is the library's)")
    ap.add_argument("--engine", default="default", choices=["default", "fused", "two_stage", "stockham"],
                    help="FFT engine of the timed context (profiling aid; the default is the library's)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def mock_seed(rank, phase, i):
    """Seed of the i-th mock a rank draws in a phase (0 warm-up, 1 timed, 2 end to end, 3 batch
    setup, 4 + r batch replay r): disjoint across ranks and phases for i < 10^5."""
    return 10 ** 7 * (rank + 1) + 10 ** 5 * phase + i


def reduce_max(x, dist):
    """Maximum of x over the ranks of the default process group (x itself on one rank)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" == r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --- CPU side: the oracle ---------------------------------------------------------------------

def oracle_sample(seed=1):
    """One oracle mock on a bounded sub-volume of the workload: 32^3 particles on a 64^3 mesh in a
    64 Mpc/h box (same 2 Mpc/h particle spacing and N_m = 2 N_p as the 512^3 / 1024 Mpc/h case),
    2LPT at z = 9, 10 COLA steps, 100-bin P(k). Returns (particle-updates, seconds)."""
    from oracle import cola, cosmology, power
    kw = workloads.COSMO
    t0 = time.perf_counter()
    r = cola.Run(64.0, 32, 64, kw["omega_m"], 9.0, 0.0, 10)
    r.make_ics(seed, cosmology.linear_pk(kw["omega_m"], kw["h"], kw["n_s"], kw["sigma8"]))
    r.run()
    power.power_from_positions(r.x, 64.0, 32, 64, 100)
    return 32 ** 3 * 10, time.perf_counter() - t0


def _oracle_worker(seed):
    return oracle_sample(seed)


def _oracle_import(_):
    from oracle import cola, cosmology, power  # noqa: F401
    return 0


def oracle_pool_run(seeds):
    """Oracle mocks of the given seeds on all host cores: one single-threaded process per core
    (spawned, so no process inherits CUDA state). Returns (particle-updates, wall seconds, cores)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"                    # inherited by the spawned workers: one thread each
    with mp.get_context("spawn").Pool(min(cores, len(seeds))) as pool:
        pool.map(_oracle_import, range(min(cores, len(seeds))))          # imports outside the clock
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, seeds)
        wall = time.perf_counter() - t0
    return sum(u for u, _ in res), wall, min(cores, len(seeds))


def cpu_baseline(budget_s=20.0):
    """The oracle as it stands on the host cores: all cores (one process each, the reported value)
    and, for reference, one core."""
    ups1, secs1 = oracle_sample(seed=999)
    cores = os.cpu_count() or 1
    per_core = max(1, min(4, int(budget_s / max(secs1, 1e-3) / 2)))
    ups, wall, used = oracle_pool_run([1000 + i for i in range(per_core * cores)])
    return {"value": ups / wall, "unit": "particle-updates/s", "cores": used, "kind": "oracle",
            "single_core_value": ups1 / secs1,
            "sample": f"{per_core * cores} oracle mocks of 32^3 particles / 64^3 mesh / 64 Mpc/h (2LPT, 10 COLA "
                      f"steps, P(k)) on {used} processes (one per host core, single-threaded numpy FP64), "
                      f"{wall:.1f} s wall; same particle spacing and mesh ratio as the 512^3 / 1024^3 workload"}


def run_reference(args, rank, world):
    """The oracle on all host cores: each step is one oracle mock per core (a bounded sub-volume of
    the workload), run concurrently; warm-up steps run the same way untimed."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for w in range(args.warmup):
        oracle_pool_run([7 + w] * cores)
    ups, secs, used = 0, 0.0, cores
    for i in range(args.steps):
        u, s, used = oracle_pool_run([100 + cores * i + j for j in range(cores)])
        ups += u
        secs += s
    v = ups / secs
    line = {"impl": "reference", "metric": "particle-updates/s per COLA step", "value": v,
            "unit": "particle-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": "32^3 particles / 64^3 mesh / 64 Mpc/h sub-volume"},
            "cpu_baseline": {"value": v, "unit": "particle-updates/s", "cores": used, "kind": "oracle",
                             "sample": f"{args.steps} steps of {used} concurrent oracle mocks (one per host core) "
                                       f"of 32^3 / 64^3 / 64 Mpc/h"},
            "e2e": {"value": v, "unit": "particle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- GPU side ---------------------------------------------------------------------------------

def batch_params(C, base_seed=1000):
    """64 uneven mocks: N_p = 64 + 32 (r mod 5), N_m = 2 N_p, L = 128 + 96 (r mod 5) Mpc/h, 10 steps."""
    out = []
    for r in range(64):
        k = r % 5
        npp = 64 + 32 * k
        out.append(C.default_params(np=npp, nm=2 * npp, box=128.0 + 96.0 * k, seed=base_seed + r,
                                    **{x: workloads.COSMO[x] for x in ("omega_m", "h", "n_s", "sigma8")}))
    return out


def run_batch(C, stream, rank, args, world=1, dist=None):
    """Mocks/hour of the 64-mock uneven batch: one CUDA graph per batch, replayed with new seeds;
    with several ranks each replays its own batch and the figures are for the whole job."""
    params = batch_params(C)
    ups = sum(p.np ** 3 * p.n_steps for p in params)
    b = C.colapm_batch_create(params, nstreams=0, stream=stream.cuda_stream)
    try:
        t0 = time.perf_counter()
        C.colapm_batch_run(b, 64, 100, seeds=[mock_seed(rank, 3, i) for i in range(64)])   # capture + stream choice
        setup = time.perf_counter() - t0
        reps = 2
        t0 = time.perf_counter()
        for rep in range(reps):
            C.colapm_batch_run(b, 64, 100, seeds=[mock_seed(rank, 4 + rep, i) for i in range(64)])
        secs = reduce_max((time.perf_counter() - t0) / reps, dist)
        hbm, src = peaks()
        achieved = (ALG_BYTES_PARTICLE + 8 * ALG_BYTES_CELL) * ups / secs / 1e9
        return {"workload": "64 mocks, N_p = 64..192 (step 32), N_m = 2 N_p, L = 128..512 Mpc/h, 10 COLA steps, "
                            "2LPT ICs + 100-bin P(k) each; one CUDA graph, new seeds per replay",
                "mocks_per_hour": 64 * world * 3600.0 / secs, "ms_per_batch": 1e3 * secs,
                "particle_updates_per_s": ups * world / secs, "worker_streams": C.colapm_batch_streams(b),
                "first_run_s_incl_capture_and_tuning": setup,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_source": f"{src} hbm_gbs",
                             "model": "736 B per particle-update (96 B/particle + 8 cells x 80 B) over the whole "
                                      "batch time, ICs and P(k) included"}}
    finally:
        C.colapm_batch_destroy(b)


def cufft_comparison(nm, box, stream, reps=3):
    """The FFT stage of one force computation with cuFFT (through torch.fft) on the same N_m^3 mesh,
    as a comparison: r2c of a real field, the spectral operator i k_j / (k^2 W) per component (W the
    CIC window, zero at k = 0), three c2r. CUDA-event times on `stream`, best of `reps`: the four
    transforms alone, and the whole stage with torch's elementwise multiplies."""
    import torch
    with torch.cuda.stream(stream):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        delta = torch.randn((nm, nm, nm), device="cuda", dtype=torch.float32, generator=gen)
        kf = 2.0 * math.pi / box
        n_full = torch.fft.fftfreq(nm, 1.0 / nm, device="cuda", dtype=torch.float32)
        n_half = torch.fft.rfftfreq(nm, 1.0 / nm, device="cuda", dtype=torch.float32)

        def sinc2(v):
            x = math.pi * v / nm
            return torch.where(v == 0, torch.ones_like(x), (torch.sin(x) / torch.where(v == 0, torch.ones_like(x), x)) ** 2)
        kz, ky, kx = (n_full * kf).view(-1, 1, 1), (n_full * kf).view(1, -1, 1), (n_half * kf).view(1, 1, -1)
        k2 = kz * kz + ky * ky + kx * kx
        win = sinc2(n_full).view(-1, 1, 1) * sinc2(n_full).view(1, -1, 1) * sinc2(n_half).view(1, 1, -1)
        green = torch.where(k2 > 0, 1.0 / (k2 * win), torch.zeros_like(k2))
        del k2, win
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

        def once():
            ev[0].record(stream)
            dk = torch.fft.rfftn(delta)
            for _ in range(3):
                torch.fft.irfftn(dk, s=(nm, nm, nm))
            ev[1].record(stream)
            dk = torch.fft.rfftn(delta)
            dk *= green
            for kv in (kx, ky, kz):
                torch.fft.irfftn(dk * (1j * kv), s=(nm, nm, nm))
            ev[2].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        once()                                    # plans and workspace
        t = [once() for _ in range(reps)]
    res = {"transforms_ms": min(a for a, _ in t), "stage_ms": min(b for _, b in t)}
    del delta, green
    torch.cuda.empty_cache()
    return res


# forward FLOPs per voxel of the 3-16-16-16-3 network with 3^3 taps (true channel counts)
NN_FLOP_VOXEL = 2 * 27 * (3 * 16 + 16 * 16 + 16 * 16 + 16 * 3)


def run_learned(C, stream, rank, train_steps=3000):
    """The learned correction on 128^3 particles in 256 Mpc/h: coarse = 128^3 mesh, 5 steps; fine =
    384^3 mesh, 50 steps; 256 seeds, 224 to train and 32 to test; one Adam step per pair draw."""
    import torch
    from paper_1506_03737_gb300 import learned
    pc, pf = learned.pair_params(128, 256.0, 128, 5, 384, 50,
                                 {x: workloads.COSMO[x] for x in ("omega_m", "h", "n_s", "sigma8")})
    seeds = [100000 * rank + s for s in range(256)]
    t0 = time.perf_counter()
    pairs = learned.Pairs(pc, pf, seeds, nbins=24, stream=stream.cuda_stream)
    gen = time.perf_counter() - t0
    train_idx, test_idx = list(range(224)), list(range(224, 256))
    s_in, s_out = pairs.scales(train_idx)
    net = C.colapm_nn_create(128, C.nn_default_config(s_in=s_in, s_out=s_out, lr=1e-3, seed=1), stream.cuda_stream)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        learned.train(net, pairs, train_idx, train_steps, seed=rank)
        train_s = time.perf_counter() - t0
        res = learned.evaluate(net, pairs, test_idx, cross_seeds=4)
        # forward (inference) time with CUDA events on the network's stream
        out = torch.empty_like(pairs.coarse[0])
        for _ in range(3):
            C.colapm_nn_forward(net, pairs.coarse[0], out)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        ev0.record(stream)
        for _ in range(reps):
            C.colapm_nn_forward(net, pairs.coarse[0], out)
        ev1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = ev0.elapsed_time(ev1) / reps
        tf = NN_FLOP_VOXEL * 128 ** 3 / (fwd_ms / 1e3) / 1e12
        _, peak_src = peaks()
        tpeak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"] \
            if peak_src == "measured" else 1700.0
        per_coarse = pairs.secs["coarse"] / len(seeds)
        per_fine = pairs.secs["fine"] / len(seeds)
        r_hi = lambda r: float(np.nanmean(r[len(r) // 2:]))          # noqa: E731
        return {
            "workload": "128^3 particles, L = 256 Mpc/h; coarse 128^3 mesh 5 COLA steps, fine 384^3 mesh "
                        "50 steps, same seeds; net 3-16-16-16-3 periodic 3^3 convs, BF16 x BF16 -> FP32",
            "pairs": len(seeds), "train_pairs": len(train_idx), "test_pairs": len(test_idx),
            "pair_generation_s": gen, "train_steps": train_steps, "train_ms_per_step": 1e3 * train_s / train_steps,
            "forward_ms": fwd_ms,
            "pk_err_plain": res["pk_err_plain"], "pk_err_net": res["pk_err_net"],
            "mse_plain_mpc2": res["mse_plain"], "mse_net_mpc2": res["mse_net"],
            "r_high_k_plain": r_hi(res["r_plain"]), "r_high_k_net": r_hi(res["r_net"]),
            "mocks_per_hour_coarse_plus_net": 3600.0 / (per_coarse + fwd_ms / 1e3),
            "mocks_per_hour_fine": 3600.0 / per_fine,
            "note": "pk_err = mean over 24 log k-bins below the particle Nyquist frequency of |<P>/<P_fine> - 1| "
                    "on the 32 test seeds, all spectra on the 128^3 mesh; r_high_k = mean cross-correlation with "
                    "the fine density over the upper 12 bins (4 test seeds)",
            "conv_roofline": {"bound": "tensor", "kernel": "forward (4 conv launches + input pack)",
                              "achieved": tf, "peak": tpeak, "unit": "TFLOP/s", "frac": tf / tpeak,
                              "flop_per_voxel": NN_FLOP_VOXEL, "peak_source": f"{peak_src} bf16_tflops_sustained"},
        }
    finally:
        C.colapm_nn_destroy(net)
        pairs.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_1506_03737_gb300 import colapm as C

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(x, dist)

    kw = workloads.run_params(args.workload)
    np_, nm, nsteps = kw["np"], kw["nm"], kw["n_steps"]
    stream = torch.cuda.Stream()
    ctx = C.colapm_create(C.default_params(**kw), stream.cuda_stream)
    if args.engine != "default":   # (fused x-y bits, two-stage) as colapm_set_engine takes them
        fused, two = {"fused": (3, 1), "two_stage": (0, 1), "stockham": (0, 0)}[args.engine]
        C.colapm_set_engine(ctx, fused, two, 256)
    if args.sort is not None:
        C.colapm_set_sort(ctx, args.sort)
    if args.sort_tiles is not None:
        C.colapm_set_sort_tiles(ctx, args.sort_tiles)
    if args.deposit_tiles is not None:
        C.colapm_set_deposit_tiles(ctx, args.deposit_tiles)
    nbins = 100
    kd = torch.empty(nbins, dtype=torch.float64, device="cuda")
    pd = torch.empty(nbins, dtype=torch.float64, device="cuda")
    nd = torch.empty(nbins, dtype=torch.int64, device="cuda")

    def mock(seed, k_out, p_out, n_out):
        C.colapm_reseed(ctx, seed)
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        C.colapm_power(ctx, nbins, 0.0, 0.0, k_out, p_out, n_out)

    for w in range(args.warmup):
        mock(mock_seed(rank, 0, w), kd, pd, nd)
    C.colapm_get_timing(ctx)                     # clear
    C.colapm_set_timing(ctx, True)
    launches0 = C.colapm_kernel_launches(ctx)

    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for s in range(args.steps):
            mock(mock_seed(rank, 1, s), kd, pd, nd)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    launches = C.colapm_kernel_launches(ctx) - launches0
    phase_ms, phase_n = C.colapm_get_timing(ctx)
    C.colapm_set_timing(ctx, False)

    updates = np_ ** 3 * nsteps * args.steps * world
    value = job_value(np_ ** 3 * nsteps * args.steps, world, ms_max)

    # end to end: host buffers through the public C calls, the step's result read back to host
    e2e = None
    if not args.no_e2e:
        kh = torch.empty(nbins, dtype=torch.float64, pin_memory=True)
        ph = torch.empty(nbins, dtype=torch.float64, pin_memory=True)
        nh = torch.empty(nbins, dtype=torch.int64, pin_memory=True)
        posh = torch.empty((np_ ** 3, 3), dtype=torch.float32, pin_memory=True)
        momh = torch.empty((np_ ** 3, 3), dtype=torch.float32, pin_memory=True)
        # the catalogue copy of one mock overlaps the next mock (copy stream, device staging array)
        mock(mock_seed(rank, 3, 0), kh, ph, nh)      # untimed: allocates the staging array
        C.colapm_get_particles_async(ctx, posh, momh)
        C.colapm_wait_particles(ctx)
        barrier()
        t0 = time.perf_counter()
        for s in range(args.steps):
            mock(mock_seed(rank, 2, s), kh, ph, nh)
            C.colapm_get_particles_async(ctx, posh, momh)
        C.colapm_wait_particles(ctx)
        torch.cuda.synchronize()
        barrier()
        secs = max_over_ranks(time.perf_counter() - t0)
        d2h = nbins * 24 + posh.numel() * 4 + momh.numel() * 4
        e2e = {"value": updates / secs, "unit": "particle-updates/s", "h2d_bytes_per_step": 8,
               "d2h_bytes_per_step": d2h,
               "note": "inputs are the seed and parameters (8 B per mock); outputs are P(k) and the final "
                       "particle catalogue (positions and momenta, float32 xyz) copied to pinned host memory, "
                       "each mock's catalogue copy overlapping the next mock; all copies landed before the "
                       "clock stops"}

    hbm, peak_src = peaks()
    roof = roofline(phase_ms, phase_n, np_, nm, hbm)
    roof["peak_source"] = f"{peak_src} hbm_gbs"
    alg_step = ALG_BYTES_PARTICLE * np_ ** 3 + ALG_BYTES_CELL * nm ** 3

    line = {
        "metric": "particle-updates/s per COLA step", "value": value, "unit": "particle-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "np": np_, "nm": nm, "box_mpc_h": kw["box"], "cola_steps": nsteps,
                   "step": "2LPT ICs + 10 COLA steps + 100-bin P(k), new seed each step",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (particle state and meshes ~35 GB)"},
        "gpu_launches": int(launches),
        "roofline": roof,
        # all step phases over the steps (P(k) times its deposit and forward passes as its own phase)
        "cola_step_ms": sum(phase_ms[p] for p in STEP_PHASES) / max(int(phase_n["gather"]), 1),
        "cola_step_roofline_frac": None,
        "phase_ms_per_mock": {k: v / args.steps for k, v in phase_ms.items()},
        "clocks": clk.summary(),
    }
    step_ms = line["cola_step_ms"]
    line["cola_step_roofline_frac"] = alg_step / (step_ms / 1e3) / 1e9 / hbm
    if e2e:
        line["e2e"] = e2e
    C.colapm_destroy(ctx)
    if not args.no_cufft and rank == 0:
        ours = sum(phase_ms[p] for p in ("fft_fwd", "poisson", "fft_inv", "fft_inv_x")) / max(int(phase_n["gather"]), 1)
        cf = cufft_comparison(nm, kw["box"], stream)
        line["cufft_comparison"] = {
            "mesh": nm, "ours_fft_stage_ms": ours, "cufft_transforms_ms": cf["transforms_ms"],
            "cufft_stage_ms": cf["stage_ms"],
            "note": "one force computation's FFT stage: ours = forward x/y passes + z pass with the Green's "
                    "function, gradient and deconvolution + inverse y and x passes (from the int64 density to "
                    "the three real force meshes); cuFFT through torch.fft: r2c of an FP32 field + 3 c2r "
                    "(transforms), and with torch's elementwise operator multiplies (stage)"}
    if not args.no_batch:
        line["batch"] = run_batch(C, stream, rank, args, world, dist)
    if not args.no_study and rank == 0:
        from paper_1506_03737_gb300 import studies
        t0 = time.perf_counter()
        res = studies.run(256, 512.0, seeds=(1, 2), stream=stream.cuda_stream,
                          cosmo={x: workloads.COSMO[x] for x in ("omega_m", "h", "n_s", "sigma8")})
        line["accuracy_study"] = {
            "workload": "256^3 particles, L = 512 Mpc/h, z 9 -> 0, 10 steps per variant, seeds 1 and 2; reference: "
                        "COLA modified lin-a 50 steps on N_m = 512; all spectra on the 512^3 mesh, 24 log bins to "
                        "the particle Nyquist frequency",
            "seconds": time.perf_counter() - t0, "variants": studies.summary(res)}
    if not args.no_learned and rank == 0:   # one training run; the other ranks have nothing to add
        line["learned"] = run_learned(C, stream, rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
