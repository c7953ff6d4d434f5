"""Benchmark: fast aperture-mass maps on one GB300 (or N, one process each).

Headline workload (the paper's image size, Sec. 5.1): a batch of 1024 x 1024
fp32 shear maps -> Kaiser-Squires -> starlet J = 7 (bands theta = 2..64 px +
smooth array), through fm_map_starlet.  Metric: Mpix*scales/s
= n^2 * J * maps / s / 1e6 (J counts arrays including the smooth one).

One JSON line on rank 0 with the headline, the roofline of the dominant
kernel, the end-to-end number through the host-buffer entry point, clocks,
the CPU oracle baseline, and side legs: the plain per-map FP64 form, the
direct M_ap comparison path per aperture radius (GPU analogue of Fig. 4) and
the batched noise maps (R realisations).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "starlet Map Mpix*scales/s, batched FP32 vs plain FP64 (<=1e-5 err); %HBM; p99 ms"
UNIT = "Mpix*scales/s"
L2_BYTES = 129 * 2 ** 20

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # unit counts x maximum SM clock
SERVE_REQUESTS = [200, 60]  # serving trace length and requests per swept rate (set from the command line)


def disc_taps(R):
    """Lattice offsets d with 0 < |d| <= R: the taps of the direct sum."""
    Ri = int(np.floor(R))
    return sum(2 * int(np.floor(np.sqrt(R * R - dy * dy))) + 1 for dy in range(-Ri, Ri + 1)) - 1


def algo_bytes_per_px_launch(kernel, fuse, ks_real=False, one_pass=False):
    """Algorithmic bytes per map pixel that one launch of `kernel` moves
    (fp32): what the kernel must read and write once.  FFT passes move
    complex maps (the real-output inverse: the column pass writes, and the
    row inverse reads, the half spectrum, 4 B/px); the KS row passes the real
    shear / convergence; the tile kernel reads kappa and writes `fuse` bands
    + c_fuse; a large scale's row pass reads c and writes r; its column pass
    reads r and c and writes c and w_j (one pass per scale: reads c, writes c
    and w_j); the fused column + next-row kernel also writes the next r."""
    return {
        "fft_rows_fwd": 8 + 8,
        "fft_cols_ks": 8 + (4 if ks_real else 8),
        "fft_rows_inv": (4 if ks_real else 8) + 4,
        "starlet_tile": 4 + 4 * fuse + 4,
        "starlet_row": 4 + 4,
        "starlet_col": (4 + 4 + 4) if one_pass else (4 + 4 + 4 + 4),
        "starlet_colrow": 4 + 4 + 4 + 4 + 4,
    }[kernel]


# ---------------------------------------------------------------------------
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel, field="dram_bytes_per_px", shape=None):
    """Bytes per map pixel of one launch of `kernel` from the committed ncu
    summary (a warm capture on a small case): DRAM read + write
    (dram_bytes_per_px) or SM <-> L2 read + write (l2_bytes_per_px), valid
    only while the kernel source is unchanged (sha at capture); None
    otherwise."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = dict(kv.split("=", 1) for kv in line.split())
        if parts.get("kernel") == kernel:
            rec = parts
    if not rec or field not in rec:
        return None
    if shape is not None and (rec.get("n"), rec.get("J"), rec.get("fuse")) != tuple(str(v) for v in shape):
        return None  # captured on another workload
    src = os.path.join(ROOT, "paper_1204_4293_gb300", "csrc", rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if sha != rec.get("sha"):
        return None
    return float(rec[field])


# Method bytes per map pixel of the fast path (fp32), the algorithmic traffic
# of the steps: Kaiser-Squires reads gamma1, gamma2 and writes kappa (12 B);
# the starlet reads kappa and writes J arrays (4 (J + 1) B); one unfused large
# scale reads c_{j-1} and writes c_j and w_j (12 B); the fused tile of F
# scales reads kappa and writes F bands and c_F (8 + 4 F B).  The floor is
# what must cross HBM at all: the shear in, the J arrays out (8 + 4 J B).
def method_groups(J, fuse):
    """Kernel groups of one KS + starlet step: (kernel kinds, method bytes per
    pixel per unit of work, units per map)."""
    return {
        "ks": (["fft_rows_fwd", "fft_cols_ks", "fft_rows_inv"], 12.0, 1),
        "starlet_tile": (["starlet_tile"], 8.0 + 4.0 * fuse, 1),
        "starlet_large_scale": (["starlet_row", "starlet_col", "starlet_colrow"], 12.0, J - 1 - fuse),
    }


def step_roofline(per_kind, px_step, J, fuse, ms_step, peak, peak_src, ks_real=False, l2_peak=None, n=1024):
    """The roofline of the dominant kernel group on the method bytes above,
    each group's fraction, and the whole step's.  per_kind: kind -> (device
    ms per step, launches per step), from CUDA events around each launch."""
    chunks = per_kind["fft_rows_fwd"][1]  # one row-FFT launch per chunk of maps
    shape = (n, J, fuse)  # the workload a committed ncu capture must match
    one_pass = "starlet_col" in per_kind and "starlet_row" not in per_kind  # large scales in one pass each
    groups = {}
    for name, (kinds, bpp, units) in method_groups(J, fuse).items():
        ks = [k for k in kinds if k in per_kind]
        if not ks:
            continue
        ms = sum(per_kind[k][0] for k in ks)
        # a unit launch: one chunk's pass of the group over one unit of work
        # (all of the group's kernels; a large scale is its row and column pass)
        launches = chunks * units
        bytes_step = bpp * px_step * units
        bytes_launch = bytes_step / launches
        avg_ms = ms / launches
        achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
        # the kernels' own reads and writes per unit launch (a large scale's
        # row pass 8 B/px and column pass 16 B/px through L2 or HBM)
        kern_bytes = sum(algo_bytes_per_px_launch(k, fuse, ks_real, one_pass) for k in ks) * px_step / chunks
        trf = [ncu_traffic(k, shape=shape) for k in ks]
        l2 = [ncu_traffic(k, "l2_bytes_per_px", shape) for k in ks]
        groups[name] = {"kernels": ks, "method_bytes_per_px": bpp * units, "ms_per_step": ms,
                        "launches_per_step": launches, "avg_launch_ms": avg_ms,
                        "method_bytes_per_launch": bytes_launch, "achieved_gbs": achieved, "frac": achieved / peak,
                        "traffic_per_launch": (sum(trf) * px_step / chunks) if all(
                            t is not None for t in trf) else None,
                        "l2_bytes_per_launch": (sum(l2) * px_step / chunks) if all(
                            t is not None for t in l2) else None,
                        "kernel_bytes_per_launch": kern_bytes}
    # the dominant kernel: the kind with the most device time per step; its group gets the roofline
    top = max(per_kind, key=lambda k: per_kind[k][0])
    dom = next(g for g in groups if top in groups[g]["kernels"])
    d = groups[dom]
    # SM <-> L2 traffic of the whole step (the chunks' intermediates stay in
    # L2): every launch of every kind at its captured bytes per pixel
    l2_px = [ncu_traffic(k, "l2_bytes_per_px", shape) for k in per_kind]
    l2 = None
    if l2_peak and all(v is not None for v in l2_px):
        l2_bpp = sum(v * per_kind[k][1] / chunks for v, k in zip(l2_px, per_kind))
        l2_gbs = l2_bpp * px_step / (ms_step * 1e-3) / 1e9
        l2 = {"bytes_per_px": l2_bpp, "achieved": l2_gbs, "peak": l2_peak["copy_gbs"], "unit": "GB/s",
              "frac": l2_gbs / l2_peak["copy_gbs"], "peak_source": l2_peak["source"],
              "bytes_source": "profiles/ncu_traffic.txt (lts__t_sectors_srcunit_tex read + write, warm capture)"}
    bpp_step = 12.0 + 4.0 * (J + 1)
    floor_bpp = 8.0 + 4.0 * J
    step_gbs = bpp_step * px_step / (ms_step * 1e-3) / 1e9
    return {
        "bound": "hbm", "kernel": f"{dom} ({' + '.join(d['kernels'])})", "achieved": d["achieved_gbs"],
        "peak": peak, "unit": "GB/s", "frac": d["frac"], "traffic": d["traffic_per_launch"],
        "peak_source": f"hbm_gbs ({peak_src})",
        "algorithmic_bytes_per_launch": d["method_bytes_per_launch"], "avg_launch_ms": d["avg_launch_ms"],
        "launches_per_step": d["launches_per_step"], "kernel_bytes_per_launch": d["kernel_bytes_per_launch"],
        "bytes_basis": "method bytes per pixel: KS 12, fused tile of F scales 8 + 4F, each unfused large scale 12 "
                      "(read c_{j-1}, write c_j and w_j), credited to the group's launches together; the group is "
                      "the one of the kernel kind with the most device time per step",
        "dominant_kernel": top,
        "fused_scales": fuse,
        "groups": groups,
        "step": {"method_bytes_per_px": bpp_step, "achieved": step_gbs, "frac": step_gbs / peak,
                 "floor_bytes_per_px": floor_bpp, "floor_frac": floor_bpp * px_step / (ms_step * 1e-3) / 1e9 / peak,
                 "floor_ms": floor_bpp * px_step / (peak * 1e9) * 1e3, "l2": l2},
        "timing": "CUDA events around every launch of the group's kernels on their launch stream; the same steps "
                  "launched eagerly with the chunks on one stream (graph bypassed, no kernel overlap); the step's "
                  "figures use the timed graph-replayed steps",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        win = [p for t, p in self.samples if t0 - 0.15 <= t <= t1 + 0.15]
        if not win:  # timed region shorter than the sampling period: nearest sample
            mid = 0.5 * (t0 + t1)
            win = [min(self.samples, key=lambda s: abs(s[0] - mid))[1]]
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[0]) for p in win if num(p[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in win for i in range(4) if p[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(win[0][1]),
                "power_w_max": max((num(p[2]) or 0) for p in win), "reasons": reasons, "samples": len(win)}


# ---------------------------------------------------------------------------
def make_inputs(fm, torch, n, batch, seed, dtype, distinct=None, alpha=2.0):
    """Seeded GRF shear maps (P(k) ~ k^-alpha, rms 0.02) + N(0, 0.1^2) shape
    noise, built on the device: GRF on the host, forward KS through the
    library; `distinct` different fields are repeated over the batch."""
    from paper_1204_4293_gb300 import synth
    distinct = min(batch, 8) if distinct is None else distinct
    kap = np.stack([synth.grf_kappa(n, alpha=alpha, seed=seed + i) for i in range(distinct)]).astype(np.float32)
    kd = torch.from_numpy(kap).cuda()
    g1, g2 = fm.fm_ks_forward(kd)
    reps = (batch + distinct - 1) // distinct
    g1 = g1.repeat(reps, 1, 1)[:batch].contiguous()
    g2 = g2.repeat(reps, 1, 1)[:batch].contiguous()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    g1 += 0.1 * torch.randn(g1.shape, generator=gen, device="cuda")
    g2 += 0.1 * torch.randn(g2.shape, generator=gen, device="cuda")
    return g1.to(dtype).contiguous(), g2.to(dtype).contiguous()


def cuda_time(torch, fn, reps):
    """Mean device time of fn over `reps` calls after one untimed call (which
    records any CUDA graph the call replays)."""
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# The FP64 oracle on the host cores: one process per core (started with
# spawn, so a pool opened after GPU work is safe), each holding the same
# synthetic shear map and running KS + starlet on it once per round.
_WORKER = {}


def _oracle_worker_init(n, J):
    import oracle
    from paper_1204_4293_gb300 import synth
    g1, g2 = oracle.ks_forward(synth.grf_kappa(n, seed=2))
    _WORKER.update(g1=g1, g2=g2, J=J)


def _oracle_worker_map(_):
    import oracle
    oracle.map_starlet(_WORKER["g1"], _WORKER["g2"], _WORKER["J"])
    return 1


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(n, J, procs):
    import multiprocessing
    import oracle
    oracle.build()  # compile once, before the workers load it
    ctx = multiprocessing.get_context("spawn")
    return ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(n, J))


def oracle_round(pool, procs):
    """One map per worker, all workers at once; returns the wall time."""
    t0 = time.perf_counter()
    pool.map(_oracle_worker_map, range(procs), chunksize=1)
    return time.perf_counter() - t0


def cpu_oracle_baseline(n, J, budget_s=12.0):
    """The FP64 oracle (KS + starlet) on all host cores, one map per core per
    round, timed over rounds until ~budget_s of wall time."""
    procs = host_cores()
    with oracle_pool(n, J, procs) as pool:
        oracle_round(pool, procs)  # warm-up (workers load the oracle)
        rounds, dt = 0, 0.0
        while dt < budget_s and rounds < 200:
            dt += oracle_round(pool, procs)
            rounds += 1
    maps = rounds * procs
    return {"value": n * n * J * maps / dt / 1e6, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{maps} map(s) of {n}x{n}, J={J}, KS + starlet in FP64, {procs} processes (one map each "
                      f"per round), {dt:.1f} s",
            "single_core": cpu_oracle_single_core(n, J)}


def cpu_oracle_single_core(n, J, budget_s=6.0):
    """The same oracle in this process on one core: maps one after another
    for ~budget_s of wall time."""
    import oracle
    from paper_1204_4293_gb300 import synth
    g1, g2 = oracle.ks_forward(synth.grf_kappa(n, seed=2))
    oracle.map_starlet(g1, g2, J)  # warm-up
    maps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or maps == 0:
        oracle.map_starlet(g1, g2, J)
        maps += 1
    dt = time.perf_counter() - t0
    return {"value": n * n * J * maps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{maps} map(s) of {n}x{n}, J={J}, KS + starlet in FP64, one thread, {dt:.1f} s"}


# ---------------------------------------------------------------------------
def run_reference(args):
    """--impl reference: the FP64 CPU oracle as the comparison arm, on all
    host cores (one map per core per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n, J = args.n, args.J
    procs = host_cores()
    with oracle_pool(n, J, procs) as pool:
        for _ in range(max(args.warmup, 1)):
            oracle_round(pool, procs)
        dt = sum(oracle_round(pool, procs) for _ in range(args.steps))
    value = n * n * J * procs * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{procs} {n}x{n} shear maps per step, one per host core (bounded sample of "
                                   f"the batched workload), KS + starlet J={J}", "n": n, "J": J,
                       "maps_per_step": procs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{args.steps} step(s) of {procs} map(s) of {n}x{n}, one process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def side_legs(fm, torch, n, J, g1, g2, pyr):
    """Plain FP64 form (and the batched FP32 step's error against it),
    direct M_ap per radius, batched noise maps."""
    out = {}
    # plain form: one map per launch, FP64, one scale per pass (no fusion)
    p1 = g1[0].double().contiguous()
    p2 = g2[0].double().contiguous()
    pyr64 = torch.empty(J, n, n, dtype=torch.float64, device="cuda")
    fn = lambda: fm.fm_map_starlet(p1, p2, J, fuse_depth=-1, out=pyr64)  # noqa: E731
    fn()
    ms = cuda_time(torch, fn, 5)
    # error of the batched FP32 step's first map against the plain FP64 form, per band:
    # max |w_fp32 - w_fp64| / RMS(w_fp64)
    fn()
    errs = [float((pyr[0, j].double() - pyr64[j]).abs().max() / pyr64[j].pow(2).mean().sqrt()) for j in range(J)]
    out["plain_fp64"] = {"value": n * n * J / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_map": ms,
                         "form": "one map per call, FP64, unfused (one starlet scale per pass)",
                         "fp32_err_per_band": errs, "fp32_max_err": max(errs)}
    # direct M_ap vs starlet per aperture radius (Fig. 4 analogue), fp32, one map
    s1, s2 = g1[0].contiguous(), g2[0].contiguous()
    kap, _ = fm.fm_ks_invert(s1.unsqueeze(0), s2.unsqueeze(0))
    kap = kap[0].contiguous()
    gb1, gb2 = g1[:8].contiguous(), g2[:8].contiguous()
    rows = []
    for j in range(1, J):
        theta = float(2 ** j)
        Jj = j + 1
        t_st = cuda_time(torch, lambda: fm.fm_starlet_forward(kap, Jj), 5)
        t_ks = cuda_time(torch, lambda: fm.fm_map_starlet(s1, s2, Jj), 5)
        reps = 3 if theta >= 32 else 5
        t_s98 = cuda_time(torch, lambda: fm.fm_map_direct(s1, s2, fm.FM_FILTER_S98, theta), reps)
        t_stq = cuda_time(torch, lambda: fm.fm_map_direct(s1, s2, fm.FM_FILTER_STARLET, theta), reps)
        # the direct sum is FP32-FMA bound: 4 flops per tap (A gamma1 + B gamma2)
        tf_s98 = 4.0 * disc_taps(theta) * n * n / (t_s98 * 1e-3) / 1e12
        tf_stq = 4.0 * disc_taps(2 * theta) * n * n / (t_stq * 1e-3) / 1e12
        # the Gaussian filter (JBJ04, b = 1/2) needs a cut well beyond theta
        # (Sec. 4.3): 5 theta; the paper expects it to cost about ten times
        # the polynomial filter cut at theta (Sec. 5.1)
        t_g = cuda_time(torch, lambda: fm.fm_map_direct(s1, s2, fm.FM_FILTER_JBJ04, theta, cut_over_theta=5.0),
                        2 if theta >= 32 else reps)
        tf_g = 4.0 * disc_taps(5 * theta) * n * n / (t_g * 1e-3) / 1e12
        # the same S98 sum over 8 maps in one launch (fm_map_direct_batch)
        t_b8 = cuda_time(torch, lambda: fm.fm_map_direct(gb1, gb2, fm.FM_FILTER_S98, theta), 2) / 8
        tf_b8 = 4.0 * disc_taps(theta) * n * n / (t_b8 * 1e-3) / 1e12
        rows.append({"theta_px": theta, "J": Jj, "starlet_ms": t_st, "ks_starlet_ms": t_ks,
                     "map_s98_cut_theta_ms": t_s98, "map_starletQ_cut_2theta_ms": t_stq,
                     "map_jbj04_cut_5theta_ms": t_g, "jbj04_over_s98": t_g / t_s98,
                     "speedup_vs_s98": t_s98 / t_st, "speedup_ks_starlet_vs_s98": t_s98 / t_ks,
                     "speedup_vs_jbj04": t_g / t_st,
                     "s98_tflops": tf_s98, "starletQ_tflops": tf_stq, "jbj04_tflops": tf_g,
                     "s98_alu_frac": tf_s98 / FP32_PEAK_TFLOPS, "starletQ_alu_frac": tf_stq / FP32_PEAK_TFLOPS,
                     "jbj04_alu_frac": tf_g / FP32_PEAK_TFLOPS,
                     "s98_batch8_ms_per_map": t_b8, "s98_batch8_alu_frac": tf_b8 / FP32_PEAK_TFLOPS})
    out["direct_map"] = rows
    out["direct_map_alu_peak"] = {"tflops": FP32_PEAK_TFLOPS, "source": "derived: 152 SMs x 128 FP32 lanes x 2 flops "
                                  "(FMA) x 2.07 GHz maximum SM clock"}
    # weighted direct M_ap on a field with 15 % masked (stars + a bad column)
    from paper_1204_4293_gb300 import synth
    wmask = torch.from_numpy(synth.star_mask(n, frac=0.15, seed=7).astype(np.float32)).cuda()
    mrows = []
    for theta in (4.0, 16.0, 64.0):
        reps = 3 if theta >= 32 else 5
        t_plain = cuda_time(torch, lambda: fm.fm_map_direct(s1, s2, fm.FM_FILTER_S98, theta), reps)
        t_mask = cuda_time(torch, lambda: fm.fm_map_direct_masked(s1, s2, wmask, fm.FM_FILTER_S98, theta), reps)
        mrows.append({"theta_px": theta, "filter": "S98 cut theta", "plain_ms": t_plain, "masked_ms": t_mask})
    gb1, gb2 = g1[:8].contiguous(), g2[:8].contiguous()
    t_b = cuda_time(torch, lambda: fm.fm_map_direct_masked(gb1, gb2, wmask, fm.FM_FILTER_S98, 16.0), 3)
    out["masked_direct_map"] = {"n": n, "masked_fraction": float(1 - wmask.mean().item()), "rows": mrows,
                                "batch8_theta16_ms_per_map": t_b / 8}
    # the other large-scale kernel path (all large scales in two kernels)
    pyr_b = torch.empty(g1.shape[0], J, n, n, dtype=torch.float32, device="cuda")
    alt = lambda: fm.fm_map_starlet(g1, g2, J, out=pyr_b, large_path=2)  # noqa: E731
    alt()
    ms_alt = cuda_time(torch, alt, 10)
    out["large_path_2"] = {"ms_per_step": ms_alt, "value": n * n * J * g1.shape[0] / (ms_alt * 1e-3) / 1e6}
    del pyr_b
    torch.cuda.empty_cache()
    out["large_fields"] = large_fields_leg(fm, torch)
    out["serving"] = serving_leg(fm, torch, nreq=SERVE_REQUESTS[0], sweep_nreq=SERVE_REQUESTS[1])
    # batched noise maps: R realisations of KS + starlet with FP64 accumulation
    R = 1000
    t_noise = cuda_time(torch, lambda: fm.fm_map_noise(s1, s2, J, R, seed=3), 2)
    t_kahan = cuda_time(torch, lambda: fm.fm_map_noise(s1, s2, J, R, seed=3, accum=1), 2)
    out["noise"] = {"R": R, "ms": t_noise, "value": n * n * J * R / (t_noise * 1e-3) / 1e6, "unit": UNIT,
                    "kahan_fp32_sums_ms": t_kahan}
    # the exact expectation of that variance (periodic boundary): one FFT pipeline
    t_exp = cuda_time(torch, lambda: fm.fm_map_noise_expected(s1, s2, J), 5)
    out["noise_expected"] = {"ms": t_exp, "boundary": "periodic",
                             "vs_monte_carlo_R1000": t_noise / t_exp}
    return out


def per_kernel_hbm(fm, fn, px, fuse, reps=3, ks_real=False):
    """Per kernel kind: device time per call (CUDA events around each launch,
    chunks on one stream), launches, algorithmic bytes per launch and the
    fraction of the measured HBM copy bandwidth that they reach."""
    peak, src = load_peaks()
    fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, 1)
    kinds = ["fft_rows_fwd", "fft_cols_ks", "fft_rows_inv", "starlet_tile", "starlet_row", "starlet_col",
             "starlet_colrow"]
    res = {}
    try:
        for k in kinds:
            fm.fm_profile_select(k)
            for _ in range(reps):
                fn()
            ms, cnt = fm.fm_profile_read()
            if cnt:
                res[k] = [ms / reps, cnt / reps]
    finally:
        fm.fm_profile_select(0)
        fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, -1)
    chunks = res["fft_rows_fwd"][1]
    one_pass = "starlet_col" in res and "starlet_row" not in res  # large scales in one pass each
    out = {}
    for k, (ms, cnt) in res.items():
        b = algo_bytes_per_px_launch(k, fuse, ks_real, one_pass) * px / chunks
        gbs = b * cnt / (ms * 1e-3) / 1e9
        out[k] = {"ms_per_call": ms, "launches": cnt, "algorithmic_bytes_per_launch": b, "gbs": gbs,
                  "frac_hbm": gbs / peak}
    out["peak_gbs"] = f"{peak} ({src})"
    return out


def large_fields_leg(fm, torch, J=9):
    """Large fields, batched: 16 x 4096^2 and 1 x 8192^2 fp32 maps, P(k) ~
    k^-2.5, starlet J = 9 (two distinct GRFs per size, repeated, plus shape
    noise)."""
    out = {}
    for n, B in ((4096, 16), (8192, 1)):
        g1, g2 = make_inputs(fm, torch, n, B, seed=40, dtype=torch.float32, distinct=min(B, 2), alpha=2.5)
        pyr = torch.empty(B, J, n, n, dtype=torch.float32, device="cuda")
        fn = lambda: fm.fm_map_starlet(g1, g2, J, out=pyr)  # noqa: E731
        fn()
        ms_builtin = cuda_time(torch, fn, 3)
        plan = fm.fm_autotune(n, J, B)  # autotuned tile form and fusion depth for this shape
        fn()
        ms = cuda_time(torch, fn, 3)
        out[f"{B}x{n}"] = {"ms": ms, "value": n * n * J * B / (ms * 1e-3) / 1e6, "unit": UNIT, "J": J,
                           "hbm_algorithmic_gbs": (12 + 4 * (J + 1)) * n * n * B / (ms * 1e-3) / 1e9,
                           "plan": plan, "ms_builtin_plan": ms_builtin}
        if B > 1:  # maps far larger than L2: each kernel's HBM roofline fraction
            out[f"{B}x{n}"]["per_kernel"] = per_kernel_hbm(fm, fn, n * n * B, plan["fuse_depth"],
                                                           ks_real=fm.fm_ks_real_output(n))
            out[f"{B}x{n}"]["ks_real_output"] = fm.fm_ks_real_output(n)
        del g1, g2, pyr
        torch.cuda.empty_cache()
    return out


def _serve_trace(fm, sv, reqs, gaps):
    """Submit `reqs` at the given inter-arrival gaps (busy-wait pacing) and
    wait for all; returns (ok results, span s)."""
    tickets = []
    due = time.perf_counter()
    for (g1, g2, J, pyr, R, var), gap in zip(reqs, gaps):
        due += gap
        while time.perf_counter() < due:
            pass
        tickets.append(sv.submit(g1, g2, J, pyr, R=R, seed=7, out_var=var))
    res = [sv.wait(t, 1800.0) for t in tickets]
    ok = [r for r in res if r.status == fm.FM_OK]
    span = (max(r.t_done_ns for r in ok) - min(r.t_submit_ns for r in ok)) / 1e9
    return ok, span


def _trace_stats(ok, span, offered):
    lat = np.array([(r.t_done_ns - r.t_submit_ns) / 1e6 for r in ok])
    wait = np.array([(r.t_admit_ns - r.t_submit_ns) / 1e6 for r in ok])
    return {"offered_req_per_s": offered, "ok": len(ok), "achieved_req_per_s": len(ok) / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "p50_queue_ms": float(np.percentile(wait, 50)), "span_s": span}


def serving_leg(fm, torch, seed=5, nreq=200, sweep_nreq=60, lam=200.0, budget_gb=64, slots=8,
                fracs=(0.3, 0.5, 0.7, 0.9)):
    """A seeded Poisson stream of mixed requests through the continuous-
    batching server: side in {256..4096}, J = log2(side) - 2, R in {0, 100,
    1000}.  The trace of `nreq` requests runs at the offered 200/s (far above
    what one GPU serves: the queue grows and latency is mostly waiting), then
    its first `sweep_nreq` requests at fractions of the achieved rate; the
    highest swept rate whose p99 stays within twice the longest request's
    own service time is the sustainable one.  Requests of one (side, R) class
    share a small pool of device buffers (inputs are only read; outputs are
    not checked here).  Also: the same trace with merging off, and the sum of
    each request's standalone time (the library's fp32 calls one after
    another, each class timed once) as the back-to-back reference."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([256, 512, 1024, 2048, 4096], nreq)
    Rs = rng.choice([0, 100, 1000], nreq)
    gaps = rng.exponential(1.0 / lam, nreq)
    pools, used = {}, {}
    reqs = []
    for side, R in zip(sides, Rs):
        side, R = int(side), int(R)
        key = (side, R)
        J = int(np.log2(side)) - 2
        cap = 4 if side >= 4096 else (8 if side >= 2048 else 24)
        pool = pools.setdefault(key, [])
        k = used.get(key, 0)
        used[key] = k + 1
        if len(pool) < cap:
            g1 = 0.1 * torch.randn(side, side, device="cuda")
            g2 = 0.1 * torch.randn(side, side, device="cuda")
            pyr = torch.empty(J, side, side, device="cuda")
            var = torch.empty(J - 1, side, side, dtype=torch.float64, device="cuda") if R else None
            pool.append((g1, g2, J, pyr, R, var))
        reqs.append(pool[k % cap])
    torch.cuda.synchronize()
    pix = [int(sd) ** 2 * (int(np.log2(sd)) - 2) * (1 + int(R)) for sd, R in zip(sides, Rs)]
    out = {"requests": nreq, "sweep_requests": sweep_nreq, "slots": slots, "budget_gb": budget_gb,
           "trace": f"seed {seed}, Poisson, side U{{256..4096}}, J=log2(side)-2, R U{{0,100,1000}}"}
    # each class alone, fp32, through the library's calls on one stream
    alone = {}
    for (side, R) in sorted(set((int(a), int(b)) for a, b in zip(sides, Rs))):
        g1, g2, J, pyr, _, var = pools[(side, R)][0]
        ms = cuda_time(torch, lambda: fm.fm_map_starlet(g1, g2, J, out=pyr), 2)
        if R:
            ms += cuda_time(torch, lambda: fm.fm_map_noise(g1, g2, J, R, seed=7, with_snr=False), 1)
        alone[(side, R)] = ms
    back_to_back_s = sum(alone[(int(a), int(b))] for a, b in zip(sides, Rs)) / 1e3
    longest_ms = max(alone[(int(a), int(b))] for a, b in zip(sides, Rs))
    with fm.Server(mem_budget_bytes=budget_gb << 30, max_slots=slots) as sv:
        for (side, R), ms in alone.items():  # warm every size once
            g1, g2, J, pyr, _, _ = pools[(side, R)][0]
            sv.wait(sv.submit(g1, g2, J, pyr), 120.0)
        ok, span = _serve_trace(fm, sv, reqs, gaps)
        sat = _trace_stats(ok, span, lam)
        sat["mpix_scales_per_s"] = sum(pix) / span / 1e6
        out["saturated"] = sat
        fm.fm_tune(fm.FM_TUNE_SERVE_MERGE, 1)
        try:
            ok, span = _serve_trace(fm, sv, reqs, gaps)
        finally:
            fm.fm_tune(fm.FM_TUNE_SERVE_MERGE, -1)
        out["saturated_no_merging"] = _trace_stats(ok, span, lam)
        fm.fm_tune(fm.FM_TUNE_SERVE_HEAVY, 0)
        try:
            ok, span = _serve_trace(fm, sv, reqs, gaps)
        finally:
            fm.fm_tune(fm.FM_TUNE_SERVE_HEAVY, -1)
        out["saturated_heavy_unlimited"] = _trace_stats(ok, span, lam)
        sweep = []
        sub, subg = reqs[:sweep_nreq], gaps[:sweep_nreq]
        for f in fracs:
            rate = f * sat["achieved_req_per_s"]
            ok, span = _serve_trace(fm, sv, sub, subg * (lam / rate))
            st = _trace_stats(ok, span, rate)
            st["drains"] = st["p99_ms"] <= 2 * longest_ms
            st["p99_over_longest_alone"] = st["p99_ms"] / longest_ms
            sweep.append(st)
        out["sweep"] = sweep
    drained = [st["offered_req_per_s"] for st in sweep if st["drains"]]
    out["sustainable_req_per_s"] = max(drained) if drained else None
    out["longest_request_alone_ms"] = longest_ms
    out["sustainable_rule"] = (f"p99 within twice the longest request's own service time "
                               f"({2 * longest_ms:.0f} ms) on the first {sweep_nreq} requests")
    out["back_to_back_fp32"] = {"trace_s": back_to_back_s, "req_per_s": nreq / back_to_back_s,
                                "mpix_scales_per_s": sum(pix) / back_to_back_s / 1e6,
                                "server_over_back_to_back": back_to_back_s / (nreq / sat["achieved_req_per_s"]),
                                "sample": "each (side, R) class timed once alone (fp32), summed over the trace"}
    # the contract's flat keys: the saturated trace
    out.update({k: sat[k] for k in ("offered_req_per_s", "achieved_req_per_s", "p50_ms", "p99_ms",
                                    "mpix_scales_per_s")})
    # plain-FP64 estimate of the same trace: each distinct (side, R) class timed
    # once in the plain form (one map, FP64, one starlet scale per pass; the
    # noise pass at R = 20, scaled to the class's R) and summed over the
    # trace as one request after another
    total_s = 0.0
    for (side, R), ms_alone in alone.items():
        count = sum(1 for a, b in zip(sides, Rs) if (int(a), int(b)) == (side, R))
        J = int(np.log2(side)) - 2
        g = (0.1 * torch.randn(2, side, side, device="cuda", dtype=torch.float64)).contiguous()
        pyr = torch.empty(J, side, side, dtype=torch.float64, device="cuda")
        ms = cuda_time(torch, lambda: fm.fm_map_starlet(g[0], g[1], J, fuse_depth=-1, out=pyr), 2)
        if R:
            rs = min(R, 20)
            ms += cuda_time(torch, lambda: fm.fm_map_noise(g[0], g[1], J, rs, seed=7, fuse_depth=-1,
                                                           with_snr=False), 1) * (R / rs)
        total_s += count * ms / 1e3
        del g, pyr
    del pools, reqs
    torch.cuda.empty_cache()
    out["plain_fp64_estimate"] = {"trace_s": total_s, "achieved_req_per_s": nreq / total_s,
                                  "sample": "each (side, R) class once; noise at R = 20 scaled to R"}
    return out


def cpu_oracle_configs():
    """The oracle on the other configurations, one process, reported only:
    noise maps at 1024^2, J = 7 with R = 20 (scaled to R = 1000) and one
    4096^2, J = 9 map of KS + starlet."""
    import oracle
    from paper_1204_4293_gb300 import synth
    oracle.build()
    out = {}
    g1, g2 = oracle.ks_forward(synth.grf_kappa(1024, seed=3))
    t0 = time.perf_counter()
    oracle.map_noise(g1, g2, 7, 20, seed=3, with_snr=False)
    dt = time.perf_counter() - t0
    out["noise_1024_R1000_s"] = dt * 1000 / 20
    out["noise_sample"] = f"R = 20 in {dt:.1f} s, one thread, scaled linearly to R = 1000"
    g1, g2 = oracle.ks_forward(synth.grf_kappa(4096, alpha=2.5, seed=40))
    t0 = time.perf_counter()
    oracle.map_starlet(g1, g2, 9)
    dt = time.perf_counter() - t0
    out["map_4096_J9_s"] = dt
    out["map_4096_value"] = 4096 * 4096 * 9 / dt / 1e6
    out["unit"] = UNIT
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--J", type=int, default=7)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--no-side", action="store_true", help="skip the side legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in plan (no autotuning)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests in the serving trace")
    ap.add_argument("--serve-sweep-requests", type=int, default=60, help="requests per swept rate")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving leg and print it")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    SERVE_REQUESTS[:] = [args.serve_requests, args.serve_sweep_requests]
    if args.serving_only:
        import torch
        from paper_1204_4293_gb300 import fastmap as fm
        print(json.dumps({"serving": serving_leg(fm, torch, nreq=args.serve_requests,
                                                 sweep_nreq=args.serve_sweep_requests)}), flush=True)
        return 0

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1204_4293_gb300 import fastmap as fm

    n, J, B = args.n, args.J, args.batch
    g1, g2 = make_inputs(fm, torch, n, B, seed=1000 * (rank + 1), dtype=torch.float32)
    pyr = torch.empty(B, J, n, n, dtype=torch.float32, device="cuda")
    step = lambda: fm.fm_map_starlet(g1, g2, J, out=pyr)  # noqa: E731

    # the library's autotuner picks the plan (fused depth, large-scale path,
    # tile form, chunk budget) for this shape before anything is timed
    plan = None if args.no_autotune else fm.fm_autotune(n, J, B)

    # warm-up (the first call records the batched call's CUDA graph)
    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    launches0 = fm.fm_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        dist.barrier()
    ms_step = e0.elapsed_time(e1) / args.steps
    launches = fm.fm_launch_count() - launches0
    clocks = sampler.summary(t0, t1) if sampler else None

    # per-kernel device time: the same steps launched eagerly with CUDA events
    # around every launch of one kernel kind (the graph is bypassed while a
    # kernel is selected), with the chunks on one stream so kernels do not
    # overlap and each launch's time is its own; the dominant kind gets the
    # roofline
    kinds = ["fft_rows_fwd", "fft_cols_ks", "fft_rows_inv", "starlet_tile", "starlet_row", "starlet_col",
             "starlet_colrow"]
    per_kind = {}
    prof_steps = max(3, min(args.steps, 20))
    fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, 1)
    for k in kinds:
        fm.fm_profile_select(k)
        for _ in range(prof_steps):
            step()
        ms, cnt = fm.fm_profile_read()
        if cnt:
            per_kind[k] = (ms / prof_steps, cnt / prof_steps)
    fm.fm_profile_select(0)
    fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, -1)

    t = torch.tensor([ms_step], device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    units = n * n * J * B * world  # whole-job pixel-scales per step
    value = units / (ms_max * 1e-3) / 1e6

    # end to end through the host-buffer entry point (pinned buffers)
    h1 = g1.cpu().pin_memory()
    h2 = g2.cpu().pin_memory()
    hout = torch.empty(B, J, n, n, dtype=torch.float32).pin_memory()
    e2e_step = lambda: fm.fm_map_starlet_host(h1, h2, J, hout)  # noqa: E731
    e2e_step()
    e2e_steps = max(3, min(args.steps, 20))
    e2e_ms = cuda_time(torch, e2e_step, e2e_steps)
    te = torch.tensor([e2e_ms], device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = units / (float(te.item()) * 1e-3) / 1e6

    extras = {}
    if rank == 0 and world == 1 and not args.no_side:
        extras = side_legs(fm, torch, n, J, g1, g2, pyr)
    if sampler:
        sampler.stop()

    if rank == 0:
        peak, peak_src = load_peaks()
        # the memory-side rates on this GPU: a 64 MiB working set stays in L2
        l2_rd, l2_cp = fm.fm_measure_bandwidth(64 << 20, 50)
        l2_peak = {"read_gbs": l2_rd, "copy_gbs": l2_cp,
                   "source": "measured here: fm_measure_bandwidth, 32 MiB read / copied into 32 MiB, 50 sweeps"}
        px_step = n * n * B
        fuse = fm.fm_starlet_fuse_depth(n, J)  # the plan's fused depth for this size
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B} x {n}x{n} fp32 shear maps per GPU per step -> Kaiser-Squires -> "
                                   f"starlet J={J} (theta=2..{2 ** (J - 1)} px + smooth)",
                       "n": n, "J": J, "maps_per_gpu": B, "parallelism": f"replicas x{world} (maps sharded)",
                       "plan": plan if plan else "built-in rules (--no-autotune)",
                       "l2": f"inputs larger than L2: {2 * B * n * n * 4 / 2**20:.0f} MB shear in + "
                             f"{B * J * n * n * 4 / 2**20:.0f} MB pyramid out per step"},
            "roofline": step_roofline(per_kind, px_step, J, fuse, ms_max, peak, peak_src, fm.fm_ks_real_output(n),
                                      l2_peak, n),
            "kernel_breakdown_ms_per_step": {k: v[0] for k, v in per_kind.items()},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * B * n * n * 4,
                    "d2h_bytes_per_step": B * J * n * n * 4, "ms_per_step": float(te.item()),
                    "api": "fm_map_starlet_host (pinned host buffers)"},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        line.update(extras)
        if "plain_fp64" in extras:
            line["batched_fp32_over_plain_fp64"] = value / extras["plain_fp64"]["value"]
            line["fp32_max_err_vs_plain_fp64"] = extras["plain_fp64"]["fp32_max_err"]
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_oracle_baseline(n, J)
            if not args.no_side:
                line["cpu_oracle_other_configs"] = cpu_oracle_configs()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
