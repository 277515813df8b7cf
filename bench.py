"""H-psi throughput and Davidson time-to-solution of the plane-wave Kohn-Sham Hamiltonian.

Headline workload: the 255-atom Si-like cell with one vacancy (41.04 x 41.04 x 20.52 bohr,
30 Ry, the stated FFT grid 96x96x48, 4 shifted k-points, 288 bands, 1020 projectors, 95,885
plane waves per k), the largest single-GPU workload of the method.  One step = H psi applied
to every band at every k-point (1152 band-applies) through the C ABI (qm_hpsi).  The headline
`value` is the precision form (QM_MIXED: FP32 FFT path, BF16x3 tensor-core nonlocal GEMMs);
the plain FP64 form is measured on the same cell under `forms.fp64`.  Secondary objects: the
64-atom cell (72^3, 4 k, 160 bands) in both forms, block Davidson to 1e-8 Ha on it, the batched
form (256 uneven cells, one persistent launch) and the 216-atom cell.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--davidson 0|1] [--batched 0|1] [--impl reference]

--impl reference times the FP64 CPU oracle (numpy, on every host core) on a bounded sample of
the same workload: a deliberately slow baseline, not a competitor.
Multi-GPU (torchrun, one process per GPU): every rank processes its own copy of the cell
(independent problems, no collective on the data path), "scaling": "weak".
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Hψ band-applies/s & Davidson time-to-1e-8 Ha: mixed/learned vs FP64 plain"
UNIT = "band-applies/s"
WORKLOAD = "si255_vacancy_96x96x48_4k_288b"
WORKLOAD2 = "si64_cubic_72^3_4k_160b"
N_FAMILIES = 18

# ALU peaks from SM count x per-SM FMA rate x max clock:
#   FP64: the nominal 1.25 TFLOP/s over 152 SMs at 2.07 GHz = 4 flop/clk/SM (2 DFMA/clk/SM)
#   FP32: 128 FMA/clk/SM
N_SM = 152
FLOP_PER_CLK_SM = {"fp64": 4, "mixed": 256}

# DRAM bytes per launch of a dominant kernel, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the current kernel, keyed by (kernel family, precision, workload);
# None where no capture of the current kernel exists.  The tensor-core nonlocal family launches
# the projection and the application GEMM once per k-point: its figure is their mean over one
# k-point of the 255-atom cell (1.844 GB and 1.479 GB; every k-point has the same shapes).
TRAFFIC_PER_LAUNCH = {("k_umma_bf16x3", "mixed", "si255_vac"): (1844459520 + 1478849536) // 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-bands", type=int, default=2,
                    help="--impl reference: oracle bands per host core per step")
    ap.add_argument("--cpu-baseline-bands", type=int, default=96,
                    help="cpu_baseline: oracle bands per host core in its one timed step (about 10 s)")
    ap.add_argument("--davidson", type=int, default=1, help="also time block Davidson to tol (0: skip)")
    ap.add_argument("--davidson-tol", type=float, default=1e-8)
    ap.add_argument("--batched", type=int, default=1, help="also time the batched form (0: skip)")
    ap.add_argument("--scf", type=int, default=1, help="also time a self-consistency run (0: skip)")
    ap.add_argument("--gw", type=int, default=1, help="also time GW plane-wave matrix elements (0: skip)")
    ap.add_argument("--tddft", type=int, default=1, help="also time real-time propagation steps (0: skip)")
    ap.add_argument("--large", type=int, default=1, help="also time H psi on the 216- and 255-atom cells (0: skip)")
    ap.add_argument("--profile", default="",
                    help="profiling run: only the precision form's H psi steps (projectors prepared) on the named "
                         "cell (config2, config4, config5) for --warmup + --steps steps, or 'gw' (the GW matrix "
                         "elements of the benchmark), for ncu command lines")
    ap.add_argument("--profile-k", type=int, default=0, help="--profile: k-points to use (0: all)")
    ap.add_argument("--profile-prec", default="mixed", choices=["mixed", "fp64"], help="--profile: precision form")
    ap.add_argument("--profile-batched", default="", help="profiling run of the batched form: mixed or fp64 "
                    "(the 256 uneven cells, the tuned shape of the benchmark, --warmup + --steps replays)")
    ap.add_argument("--davidson-255", type=int, default=1,
                    help="time Davidson on the 255-atom cell, k-point 0: the combined form vs plain FP64 (about 4 "
                         "minutes; 0: skip)")
    ap.add_argument("--davidson-255-all", type=int, default=0,
                    help="1: also solve all 4 k-points of the 255-atom cell concurrently in the combined form "
                         "(about 3 minutes)")
    ap.add_argument("--davidson-large", type=int, default=0,
                    help="1: also time Davidson on the 216-atom cell, learned vs TPA (about 2 minutes)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus = (bus_id or "").lower()
        self.proc = None
        self.path = os.path.join("/tmp", f"qm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.path)
        if not rows:
            return None
        mine = [r for r in rows if self.bus and self.bus[-12:] in r[0].lower()] or rows
        num = lambda x: x.replace(".", "").isdigit()
        sm = sorted(float(r[1]) for r in mine if num(r[1]))
        mx = max((float(r[2]) for r in mine if num(r[2])), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in mine for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(mine)}


# ------------------------------------------------------------------ oracle (CPU) leg
ORACLE_CODE = r"""
import json, sys, time
from concurrent.futures import ThreadPoolExecutor
sys.path.insert(0, ROOT)
import numpy as np
import qm_synth as S
from oracle import gspace as OG, hamiltonian as OH
cell = getattr(S, CFG)()
v = S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)
D = S.dvals(cell.nat)
nk = len(cell.kpts)
cache = {}
def setup(ik):
    if ik not in cache:
        gs = OG.gsphere(cell.lattice, cell.grid, cell.ecut_ha, cell.kpts[ik])
        cache[ik] = (gs, S.beta_of_q(gs["q"], cell.tau, cell.omega))
    return cache[ik]
pool = ThreadPoolExecutor(THREADS)
def step(i):
    ik = i % nk
    gs, beta = setup(ik)
    psi = S.psi_random(cell.seed, BANDS, len(gs["idx"]), stream=ik)
    chunks = [c for c in np.array_split(np.arange(BANDS), THREADS) if c.size]
    t = time.perf_counter()
    list(pool.map(lambda c: OH.hpsi_fft(psi[c], gs, v, beta, D), chunks))
    return time.perf_counter() - t
for i in range(min(STEPS + WARMUP, nk)):
    setup(i % nk)
times = [step(i) for i in range(WARMUP + STEPS)][WARMUP:]
print(json.dumps({"step_s": times, "bands": BANDS, "threads": THREADS}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_run(cfg, bands, threads, steps, warmup):
    """Time the FP64 oracle's H psi (oracle.hamiltonian.hpsi_fft, as it stands) on `bands`
    bands of the workload per step, the bands split over `threads` host threads (numpy's FFTs
    and one-thread BLAS release the interpreter lock).  Setup (sphere, V, projectors) is outside
    the timed steps.  Runs in a child process so that BLAS is pinned to one thread per worker."""
    code = ORACLE_CODE.replace("ROOT", repr(ROOT)).replace("CFG", repr(cfg)).replace("THREADS", str(int(threads)))
    code = code.replace("BANDS", str(int(bands))).replace("WARMUP", str(int(warmup))).replace("STEPS", str(int(steps)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode:
        raise RuntimeError("oracle leg failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(cfg, bands_per_core):
    """cpu_baseline: the oracle on every host core (bands_per_core bands per core, one timed step
    after one warm-up step) and on one core (4 bands), band-applies/s."""
    n = host_cores()
    allc = oracle_run(cfg, bands_per_core * n, n, 1, 1)
    one = oracle_run(cfg, 4, 1, 1, 0)
    v_all = allc["bands"] / allc["step_s"][0]
    v_one = one["bands"] / one["step_s"][0]
    return {"value": v_all, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{allc['bands']} bands of k-point 0 of {cfg} on {n} threads ({bands_per_core} bands per "
                      f"thread), "
                      f"FP64 numpy full-box FFT + nonlocal GEMM, {allc['step_s'][0]:.2f} s",
            "one_core": {"value": v_one, "unit": UNIT, "cores": 1,
                         "sample": f"4 bands of k-point 0, 1 thread, {one['step_s'][0]:.2f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = host_cores()
    bands = max(1, args.cpu_sample_bands) * n
    r = oracle_run("config5", bands, n, args.steps, args.warmup)
    tot = sum(r["step_s"])
    v = r["bands"] * len(r["step_s"]) / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(r["step_s"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64",
                                            "sample_bands_per_step": bands,
                                            "note": "each step: H psi on a sample of the workload's bands, "
                                                    "k-point = step mod 4"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"{bands} bands per step of {WORKLOAD}, FP64 numpy oracle on {n} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU leg
def fft_flops_per_plane(grid, nrow):
    """Algorithmic flops of one band's yz plane: 5 L log2 L per FFT of length L, both
    directions, plus the V multiply."""
    n1, n2, n3 = grid
    f = lambda L: 5.0 * L * math.log2(L)
    return 2.0 * (nrow * f(n2) + n2 * f(n3)) + 2.0 * n2 * n3


def max_over_ranks(vals, device):
    """Element-wise maximum of per-rank timings over the process group (the slowest rank
    sets the whole job's time)."""
    import torch
    t = torch.tensor([float(x) for x in vals], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t]


def read_prof(lib):
    fam = {}
    for f in range(N_FAMILIES):
        t = ctypes.c_double()
        c = ctypes.c_longlong()
        lib.qm_prof_read(f, ctypes.byref(t), ctypes.byref(c))
        if c.value:
            fam[lib.qm_prof_name(f).decode()] = {"ms_total": t.value, "launches": c.value}
    return fam


class Workload:
    """Device-resident inputs of the 64-atom cell for one precision."""

    def __init__(self, S, g, cell, rank, prec, dev):
        import numpy as np
        import torch
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        self.prec = prec
        self.psi, self.beta, self.out, self.psi_host, self.out_host, self.nrow = [], [], [], [], [], []
        for ik in range(len(cell.kpts)):
            idx, _, kpg = g.indices(ik)
            self.nrow.append(len(np.unique(idx // (cell.grid[0] * cell.grid[1]))))  # yz rows holding sticks
            p = S.psi_random(cell.seed + rank, cell.nbnd, g.npw[ik], stream=ik)
            self.psi_host.append(torch.from_numpy(p).to(cdt).pin_memory())
            self.psi.append(self.psi_host[-1].to(dev))
            self.beta.append(torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(cdt).to(dev))
            self.out.append(torch.empty_like(self.psi[-1]))
            self.out_host.append(torch.empty_like(self.psi_host[-1]).pin_memory())


def measure_hpsi(steps, warmup, Q, lib, g, cell, wl, v, D, world, dev, peaks, sample_clocks, with_e2e=True):
    import torch
    nk, nb, nproj = len(cell.kpts), cell.nbnd, cell.nproj
    stream = torch.cuda.current_stream()

    def step():
        for ik in range(nk):
            Q.qm_hpsi(g.handle, ik, wl.psi[ik], v, wl.beta[ik], D, out=wl.out[ik], prec=wl.prec, stream=stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(warmup):
        step()
    barrier()
    clocks = ClockSampler(getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", "")) if sample_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    lib.qm_prof_enable(1)
    n0 = lib.qm_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    barrier()
    launches = int(lib.qm_launch_count() - n0)
    ms = e0.elapsed_time(e1) / steps
    fam = read_prof(lib)
    lib.qm_prof_enable(0)
    clk = clocks.stop() if clocks else None

    # end to end: pinned host psi -> device, H psi, device -> pinned host, every step, through
    # the public API as a user pipelines a steady stream of steps: the input copies run on one
    # copy stream and the result copies on another, so that k-point k+1's input and k-point
    # k-1's result move while k-point k is applied.  Events order each copy with the H psi that
    # uses its buffer: k-point k's next input waits only for its own H psi of the previous step,
    # and its next H psi only for the copy-out of its previous result, so one step's copies also
    # overlap the neighbouring steps' compute.
    h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    used = [None] * nk      # H psi of k-point k done (its psi buffer free again)
    copied = [None] * nk    # copy-out of k-point k's result done (its out buffer free again)

    def e2e_step():
        ev_in = []
        for ik in range(nk):
            if used[ik] is not None:
                h2d_s.wait_event(used[ik])
            with torch.cuda.stream(h2d_s):
                wl.psi[ik].copy_(wl.psi_host[ik], non_blocking=True)
            ev_in.append(torch.cuda.Event())
            ev_in[-1].record(h2d_s)
        for ik in range(nk):
            stream.wait_event(ev_in[ik])
            if copied[ik] is not None:
                stream.wait_event(copied[ik])
            Q.qm_hpsi(g.handle, ik, wl.psi[ik], v, wl.beta[ik], D, out=wl.out[ik], prec=wl.prec, stream=stream)
            used[ik] = torch.cuda.Event()
            used[ik].record(stream)
            d2h_s.wait_event(used[ik])
            with torch.cuda.stream(d2h_s):
                wl.out_host[ik].copy_(wl.out[ik], non_blocking=True)
            copied[ik] = torch.cuda.Event()
            copied[ik].record(d2h_s)

    ems = None
    if with_e2e:
        for _ in range(2):
            e2e_step()
        barrier()
        stream.wait_stream(d2h_s)
        stream.wait_stream(h2d_s)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        h2d_s.wait_stream(stream)
        d2h_s.wait_stream(stream)
        esteps = max(3, steps // 3)
        for _ in range(esteps):
            e2e_step()
        stream.wait_stream(d2h_s)     # the timed region ends when the last result is on the host
        e3.record(stream)
        barrier()
        ems = e2.elapsed_time(e3) / esteps
    h2d = sum(t.numel() * t.element_size() for t in wl.psi_host)
    d2h = sum(t.numel() * t.element_size() for t in wl.out_host)
    if world > 1:
        ms, ems = max_over_ranks([ms, ems if ems is not None else 0.0], dev)
    band_applies = nb * nk * world

    def roofline_of(name, d):
        """Roofline of kernel family `name` from its summed CUDA-event time over the timed steps."""
        avg_ms = d["ms_total"] / d["launches"]
        per_step = d["launches"] / steps
        smax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        fl_pk = FLOP_PER_CLK_SM[wl.prec] * N_SM * smax / 1e12
        fl = None
        bound = "alu"
        extra = {}
        if name == "k_plane":
            fl = sum(nb * cell.grid[0] * fft_flops_per_plane(cell.grid, wl.nrow[ik]) for ik in range(nk))
        elif name in ("k_gemm_tn", "k_gemm_cn"):
            fl = 8.0 * nproj * nb * sum(g.npw)   # 8 flops per complex multiply-add, all k
        elif name == "k_umma_bf16x3":
            # projection + application: 8 flops per complex multiply-add each; the method (3-term
            # BF16 split) issues 6 BF16 products per FP32-accurate one, all on the tensor pipe
            useful = 2 * 8.0 * nproj * nb * sum(g.npw)
            fl = 6 * useful
            bound = "tensor"
            fl_pk = float(peaks.get("bf16_tflops_sustained", 1742.0))
            extra = {"useful_tflops": useful / per_step / (avg_ms * 1e-3) / 1e12,
                     "flops_counted": "BF16 products of the 3-term split (6 per FP32-accurate product); "
                                      "useful_tflops counts each complex multiply-add once (8 flops)"}
        if fl is None:
            return {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": None,
                    "kernel": name, "traffic": None, "avg_launch_ms": avg_ms}
        fl /= per_step
        roof = {"bound": bound, "achieved": fl / (avg_ms * 1e-3) / 1e12, "peak": fl_pk, "unit": "TFLOP/s"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof.update(extra)
        tpl = TRAFFIC_PER_LAUNCH.get((name, wl.prec, cell.name))
        roof.update({"kernel": name, "traffic": tpl, "avg_launch_ms": avg_ms, "launches_per_step": per_step,
                     "peak_source": ("measured: cuBLAS bf16 sustained, MEASURED_PEAKS.json (of measured)"
                                     if bound == "tensor" else
                                     "derived: %d SMs x %d flop/clk/SM x %.0f MHz" % (
                                         N_SM, FLOP_PER_CLK_SM[wl.prec], smax / 1e6))})
        return roof

    # roofline of the dominant kernel family (largest summed device time; in the precision form
    # the tensor-core nonlocal kernels run on the handle's second stream, concurrently with the
    # FFT kernels on the caller's stream)
    roof = roofline_of(*max(fam.items(), key=lambda kv: kv[1]["ms_total"])) if fam else None
    others = {k: roofline_of(k, d) for k, d in fam.items()
              if k in ("k_plane", "k_umma_bf16x3", "k_gemm_cn", "k_gemm_tn") and (roof is None or k != roof["kernel"])}
    out = {"value": band_applies / (ms * 1e-3), "ms_per_step": ms, "gpu_launches": launches, "kernels": fam,
           "roofline": roof, "roofline_other": others, "clocks": clk,
           "l2": "inputs larger than L2: psi %.0f MB + beta %.0f MB per step" % (
               h2d / 1e6, sum(b.numel() * b.element_size() for b in wl.beta) / 1e6)}
    if ems is not None:
        out["e2e"] = {"value": band_applies / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": ems}
    return out


def measure_fft_path(steps, warmup, Q, g, cell, wl, v, fam_live, ms_live, peaks):
    """The FFT path (scatter, stick-pruned 3D FFTs, V multiply, gather, kinetic term: K1-K3) of the
    precision form against HBM, on the fused design's bytes per band-apply: psi read twice, H psi
    written once, four passes over the stick buffer (N1 x nstick complex values per band).  Alone:
    qm_hpsi without projectors (only the FFT kernels run; without the tensor-core stream to overlap,
    the library chunks the bands so that the stick buffer stays in L2), CUDA events around the
    steps.  Live: the
    three kernels' summed event time inside the headline step, where they share the SMs with the
    tensor-core stream."""
    import numpy as np
    import torch
    nk, nb = len(cell.kpts), cell.nbnd
    cs = 8
    nbytes = 0.0
    for ik in range(nk):
        idx, _, _ = g.indices(ik)
        nstick = int(np.unique(idx // cell.grid[0]).size)
        nbytes += nb * (3.0 * g.npw[ik] * cs + 4.0 * cell.grid[0] * nstick * cs)
    stream = torch.cuda.current_stream()

    def step():
        for ik in range(nk):
            Q.qm_hpsi(g.handle, ik, wl.psi[ik], v, None, None, out=wl.out[ik], prec="mixed", stream=stream)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pk = peaks.get("hbm_gbs")
    out = {"bytes_per_band_apply": nbytes / (nb * nk), "bytes_per_step": nbytes, "peak": pk, "unit": "GB/s",
           "alone": {"ms_per_step": ms, "achieved": nbytes / (ms * 1e-3) / 1e9}}
    out["alone"]["frac"] = out["alone"]["achieved"] / pk if pk else None
    live = sum(fam_live[k]["ms_total"] for k in ("k_stick_inverse", "k_plane", "k_stick_forward") if k in fam_live)
    if live > 0:
        lms = live / steps
        out["live"] = {"ms_per_step": lms, "achieved": nbytes / (lms * 1e-3) / 1e9}
        out["live"]["frac"] = out["live"]["achieved"] / pk if pk else None
    return out


def run_davidson(args, Q, lib, g, cell, wl64, v, D):
    """Block Davidson to args.davidson_tol at every k-point from the seeded random start:
    the plain FP64 form, FP64 with 10 % buffer bands (only the lowest 160 must converge), the
    precision form (QM_MIXED) with the buffer bands, and the same with the 4 k-point solves run
    concurrently (qm_davidson_batched).  Wall time of the calls."""
    import numpy as np
    import torch

    import qm_synth as S
    nk, nb = len(cell.kpts), cell.nbnd
    out = {"tol_ha": args.davidson_tol, "nbnd": nb, "nk": nk}
    eigs = {}
    nextra = max(1, nb // 10)
    for form, prec, extra in (("fp64", "fp64", 0), ("fp64_buffer", "fp64", nextra), ("mixed_buffer", "mixed", nextra)):
        per_k = []
        lib.qm_prof_enable(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ik in range(nk):
            p = torch.from_numpy(S.psi_random(cell.seed, nb + extra, g.npw[ik], stream=ik)).cuda()
            eig, info = Q.qm_davidson(g.handle, ik, p, v, wl64.beta[ik], D, tol=args.davidson_tol, max_iter=300,
                                      raise_not_converged=False, prec=prec, nconv=nb)
            eigs.setdefault(form, []).append(eig[:nb])
            rec = {k: info[k] for k in ("iterations", "iterations_mixed", "band_applies", "band_applies_mixed",
                                        "max_residual", "converged", "seconds")}
            h = info["history"]
            rec["history_every_10"] = [h[i] for i in range(0, len(h), 10)]
            per_k.append(rec)
        torch.cuda.synchronize()
        out[form] = {"seconds_total": time.perf_counter() - t0, "nbnd_solved": nb + extra, "per_k": per_k,
                     "kernels": read_prof(lib)}
        lib.qm_prof_enable(0)
    # the batched form: the 4 k-point solves of the buffered precision form run concurrently
    # (qm_davidson_batched, one stream and workspace each)
    jobs = []
    for ik in range(nk):
        p = torch.from_numpy(S.psi_random(cell.seed, nb + nextra, g.npw[ik], stream=ik)).cuda()
        jobs.append({"g": g.handle, "ik": ik, "psi": p, "vloc": v, "beta": wl64.beta[ik], "D": D})
    lib.qm_prof_enable(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = Q.qm_davidson_batched(jobs, tol=args.davidson_tol, max_iter=300, prec="mixed", nconv=nb,
                                raise_not_converged=False)
    torch.cuda.synchronize()
    out["mixed_buffer_batched"] = {
        "seconds_total": time.perf_counter() - t0, "nbnd_solved": nb + nextra, "concurrent_jobs": nk,
        "per_k": [{k: info[k] for k in ("iterations", "iterations_mixed", "band_applies", "max_residual", "converged",
                                        "seconds")} for _, info in res],
        "kernels": read_prof(lib)}
    lib.qm_prof_enable(0)
    eigs["mixed_buffer_batched"] = [eig[:nb] for eig, _ in res]
    for form in ("fp64_buffer", "mixed_buffer", "mixed_buffer_batched"):
        out[f"speedup_{form}_vs_fp64"] = out["fp64"]["seconds_total"] / out[form]["seconds_total"]
        out[f"max_eig_diff_{form}_vs_fp64_ha"] = float(max(np.abs(a - b).max()
                                                         for a, b in zip(eigs["fp64"], eigs[form])))
    # the same buffer bands on both sides: the precision and batched forms' own gain
    for form in ("mixed_buffer", "mixed_buffer_batched"):
        out[f"speedup_{form}_vs_fp64_buffer"] = out["fp64_buffer"]["seconds_total"] / out[form]["seconds_total"]
    return out


def product_grid(Q, cell):
    """FFT grid the library's rule gives a cell (a throw-away Gamma-point gspace)."""
    g = Q.GSpace(cell.lattice, [[0.0, 0.0, 0.0]], cell.ecut_ha, None)
    grid = tuple(g.grid)
    g.close()
    return grid


def run_batched(args, Q, S, dev):
    """The batched form: 256 uneven cells (2-16 atoms, 15-30 Ry, grids 18^3-48^3, 8-48 bands,
    1-8 k-points) as one persistent launch replayed from a CUDA graph (shape autotuned),
    against the per-cell loop of qm_hpsi calls, in both precisions."""
    import torch
    cells = S.config3_cells(lambda c: product_grid(Q, c))
    out = {"workload": "256 uneven Si-like cells (2-16 atoms, 15-30 Ry, grids 18^3-48^3, 8-48 bands, 1-8 k)"}
    stream = torch.cuda.current_stream()
    for prec in ("mixed", "fp64"):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        gss, jobs = [], []
        for cell in cells:
            g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
            gss.append(g)
            v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid, cell.depth, cell.width,
                                                ortho_period=cell.ortho_period)).to(dev)
            D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
            for ik in range(len(cell.kpts)):
                _, _, kpg = g.indices(ik)
                psi = torch.from_numpy(S.psi_random(cell.seed, cell.nbnd, g.npw[ik], stream=ik)).to(cdt).to(dev)
                beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega, cell.rc)).to(cdt).to(dev)
                jobs.append({"g": g.handle, "ik": ik, "psi": psi, "vloc": v, "beta": beta, "D": D,
                             "out": torch.empty_like(psi)})
        t0 = time.time()
        b = Q.Batch(jobs, prec=prec, stream=stream)
        tune_s = time.time() - t0
        info = b.info()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(max(3, args.warmup)):
            b.run(stream)
        torch.cuda.synchronize()
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            b.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        b.check(stream)
        ms = e0.elapsed_time(e1) / reps

        def loop():
            for j in jobs:
                Q.qm_hpsi(j["g"], j["ik"], j["psi"], j["vloc"], j["beta"], j["D"], out=j["out"], prec=prec,
                          stream=stream)
        for _ in range(2):
            loop()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            loop()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_loop = e0.elapsed_time(e1) / 3
        ba = info["band_applies"]
        out[prec] = {"value": ba / ms * 1e3, "unit": UNIT, "ms_per_replay": ms, "band_applies": ba,
                     "jobs": len(jobs), "launches_per_replay": 1,
                     "per_cell_loop": {"value": ba / ms_loop * 1e3, "ms": ms_loop},
                     "speedup_vs_loop": ms_loop / ms, "shape": {k: info[k] for k in (
                         "ctas_per_sm", "item_points", "group_mb", "grid", "items", "smem_bytes", "candidates")},
                     "autotune_s": tune_s, "device_bytes": info["device_bytes"]}
        b.close()
        del jobs
        for g in gss:
            g.close()
        torch.cuda.empty_cache()
    return out


def run_large_cells(args, Q, S, dev):
    """H psi throughput (both precisions) on the 216-atom displaced cube (90^3, 480 bands,
    Gamma): one warm-up step, then timed steps with CUDA events; the states are real in real
    space, and the Gamma-point form (qm_hpsi_gamma, two bands per FFT) is timed beside qm_hpsi."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for cell in (S.config4(),):
        g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
        v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
        D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
        rec = {"grid": list(cell.grid), "nat": cell.nat, "nbnd": cell.nbnd, "nk": len(cell.kpts), "npw": g.npw,
               "nproj": cell.nproj}
        host = []
        for ik in range(len(cell.kpts)):
            _, mil, kpg = g.indices(ik)
            host.append((torch.from_numpy(S.psi_random_real(cell.seed, cell.nbnd, mil, stream=ik)),
                         torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega))))
        for form, steps in (("mixed", 5), ("fp64", 1), ("mixed_gamma", 5), ("fp64_gamma", 2)):
            prec = form.split("_")[0]
            cdt = torch.complex128 if prec == "fp64" else torch.complex64
            psi = [h[0].to(dev).to(cdt) for h in host]
            beta = [h[1].to(dev).to(cdt) for h in host]
            outs = [torch.empty_like(p) for p in psi]
            apply = Q.qm_hpsi_gamma if form.endswith("gamma") else Q.qm_hpsi

            def step():
                for ik in range(len(cell.kpts)):
                    apply(g.handle, ik, psi[ik], v, beta[ik], D, out=outs[ik], prec=prec, stream=stream)
            step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            rec[form] = {"value": cell.nbnd * len(cell.kpts) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                         "steps": steps}
            del psi, beta, outs
            torch.cuda.empty_cache()
        rec["mixed_over_fp64"] = rec["mixed"]["value"] / rec["fp64"]["value"]
        rec["gamma_over_complex"] = {p: rec[p + "_gamma"]["value"] / rec[p]["value"] for p in ("mixed", "fp64")}
        out[cell.name] = rec
        del host
        g.close()
    return out


def train_network(Q, S, dev):
    """The learned preconditioner trained as the library's training driver does it: samples
    from Davidson snapshots on 12 small cells of the uneven-cell generator (seed 101, disjoint
    from every workload's), 1500 full-batch Adam steps."""
    import torch
    from paper_2308_07277_gb300 import learned
    cells = [c for c in S.config3_cells(lambda c: product_grid(Q, c), n=40, seed=101)
             if c.grid[0] * c.grid[1] * c.grid[2] <= 30 ** 3][:12]
    parts = []
    t0 = time.time()
    for cell in cells:
        nb = min(cell.nbnd, 16)
        g = Q.GSpace(cell.lattice, cell.kpts[:1], cell.ecut_ha, cell.grid)
        _, _, kpg = g.indices(0)
        v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid, cell.depth, cell.width,
                                            ortho_period=cell.ortho_period)).to(dev)
        beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega, cell.rc)).to(dev)
        D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
        psi = torch.from_numpy(S.psi_random(cell.seed, nb + 8, g.npw[0], stream=0)).to(dev)
        parts += learned.collect(g.handle, 0, v, beta, D, psi, nb)
        g.close()
    ds = learned.assemble(parts)
    theta = learned.init_theta(1, dev)
    hist = learned.train(ds, theta, steps=1500, lr=1e-3)
    return theta, {"samples": int(ds[1].shape[0]), "bands": int(ds[0].numel() - 1), "loss_first": float(hist[0]),
                   "loss_last": float(hist[-1]), "seconds": time.time() - t0}


def run_davidson_large(args, Q, S, dev, theta):
    """Davidson to 1e-8 Ha on the learned-form workload (216-atom cell, 480 bands, Gamma;
    precision form with 10 % buffer bands, TPA vs the trained network)."""
    import numpy as np
    import torch
    cell = S.config4()
    g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    _, _, kpg = g.indices(0)
    v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
    beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    nb, nextra = cell.nbnd, cell.nbnd // 10
    rec, eigs = {}, {}
    for name, mlp in (("tpa", None), ("learned", theta)):
        p = torch.from_numpy(S.psi_random(cell.seed, nb + nextra, g.npw[0], stream=0)).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eig, info = Q.qm_davidson(g.handle, 0, p, v, beta, D, tol=args.davidson_tol, max_iter=300, prec="mixed",
                                  nconv=nb, mlp=mlp, raise_not_converged=False)
        torch.cuda.synchronize()
        rec[name] = {"seconds": time.perf_counter() - t0, **{k: info[k] for k in (
            "iterations", "iterations_mixed", "band_applies", "converged", "max_residual", "precond_fallback")}}
        eigs[name] = eig[:nb]
    rec["max_eig_diff_ha"] = float(np.abs(eigs["tpa"] - eigs["learned"]).max())
    g.close()
    return {cell.name: rec}


def run_davidson_255(args, Q, S, dev, theta):
    """The all-forms workload: Davidson to 1e-8 Ha on the 255-atom cell (96x96x48, 288 bands,
    1020 projectors).  k-point 0: plain FP64 (no buffer bands) against the combined form
    (precision form + 28 buffer bands + the learned preconditioner); with --davidson-255-all 1
    also the combined form on all 4 k-points solved concurrently (qm_davidson_batched).  Wall
    time of the calls."""
    import numpy as np
    import torch
    cell = S.config5()
    g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    nk, nb, nextra = len(cell.kpts), cell.nbnd, cell.nbnd // 10
    betas = []
    for ik in range(nk):
        _, _, kpg = g.indices(ik)
        betas.append(torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(dev))
    out, eigs = {"tol_ha": args.davidson_tol, "nbnd": nb}, {}
    for name, prec, extra, mlp in (("fp64", "fp64", 0, None), ("combined", "mixed", nextra, theta)):
        p = torch.from_numpy(S.psi_random(cell.seed, nb + extra, g.npw[0], stream=0)).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eig, info = Q.qm_davidson(g.handle, 0, p, v, betas[0], D, tol=args.davidson_tol, max_iter=400, prec=prec,
                                  nconv=nb, mlp=mlp, raise_not_converged=False)
        torch.cuda.synchronize()
        out[f"k0_{name}"] = {"seconds": time.perf_counter() - t0, **{k: info[k] for k in (
            "iterations", "iterations_mixed", "band_applies", "converged", "max_residual", "restarts",
            "precond_fallback")}}
        eigs[name] = eig[:nb]
        del p
    out["k0_speedup_combined_vs_fp64"] = out["k0_fp64"]["seconds"] / out["k0_combined"]["seconds"]
    out["k0_max_eig_diff_ha"] = float(np.abs(eigs["fp64"] - eigs["combined"]).max())
    if not args.davidson_255_all:
        g.close()
        return out
    jobs = [{"g": g.handle, "ik": ik, "vloc": v, "beta": betas[ik], "D": D,
             "psi": torch.from_numpy(S.psi_random(cell.seed, nb + nextra, g.npw[ik], stream=ik)).to(dev)}
            for ik in range(nk)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = Q.qm_davidson_batched(jobs, tol=args.davidson_tol, max_iter=400, prec="mixed", nconv=nb, mlp=theta,
                                raise_not_converged=False)
    torch.cuda.synchronize()
    out["all_k_combined_concurrent"] = {
        "seconds": time.perf_counter() - t0,
        "per_k": [{k: i[k] for k in ("iterations", "converged", "max_residual", "precond_fallback")} for _, i in res],
        "k0_max_eig_diff_vs_fp64_ha": float(np.abs(res[0][0][:nb] - eigs["fp64"]).max())}
    g.close()
    return out


def run_tddft(args, Q, S, dev):
    """Real-time propagation on the 255-atom cell, k-point 0, all 288 bands: ETRS steps of order 4
    (two half steps, 8 H psi applications and 8 Taylor updates per step), the precision form
    (projectors prepared) and plain FP64, CUDA events around the steps."""
    import torch
    cell = S.config5()
    g = Q.GSpace(cell.lattice, cell.kpts[:1], cell.ecut_ha, cell.grid)
    v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    _, _, kpg = g.indices(0)
    dt, order, nb = 0.05, 4, cell.nbnd
    out = {"workload": "si255_vacancy_96x96x48_k0_288b", "step": "ETRS, Taylor order %d per half step" % order,
           "dt_au": dt, "hpsi_per_step": 2 * order, "unit": "band-steps/s"}
    stream = torch.cuda.current_stream()
    for prec, steps, warm in (("mixed", 5, 2), ("fp64", 1, 1)):
        cdt = torch.complex64 if prec == "mixed" else torch.complex128
        psi = torch.from_numpy(S.psi_random(cell.seed, nb, g.npw[0], stream=0)).to(cdt).to(dev)
        beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(cdt).to(dev)
        work = torch.empty(2 * psi.numel(), dtype=cdt, device=dev)
        if prec == "mixed":
            Q.qm_hpsi_prepare(g.handle, 0, beta)
        for _ in range(warm):
            Q.qm_tddft_etrs(g.handle, 0, psi, v, v, beta, D, dt, order, prec=prec, work=work, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            Q.qm_tddft_etrs(g.handle, 0, psi, v, v, beta, D, dt, order, prec=prec, work=work, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"value": nb / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
                     "band_applies_per_s": 2 * order * nb / (ms * 1e-3)}
        if prec == "mixed":
            # the Taylor update kernel (family "other" here) against HBM: it reads and writes the new
            # term and psi, 4 complex values per element
            lib = Q.api._lib.load()
            lib.qm_prof_enable(1)
            Q.qm_tddft_etrs(g.handle, 0, psi, v, v, beta, D, dt, order, prec=prec, work=work, stream=stream)
            torch.cuda.synchronize()
            fam = read_prof(lib)
            lib.qm_prof_enable(0)
            acc = fam.get("other")
            if acc:
                avg = acc["ms_total"] / acc["launches"]
                nbytes = 4 * 8.0 * nb * g.npw[0]
                out["taylor_update_roofline"] = {
                    "kernel": "k_taylor_acc", "bound": "hbm", "achieved": nbytes / (avg * 1e-3) / 1e9,
                    "peak": load_peaks()[0].get("hbm_gbs"), "unit": "GB/s", "avg_launch_ms": avg,
                    "bytes_per_launch": nbytes, "launches_per_step": acc["launches"]}
                r = out["taylor_update_roofline"]
                r["frac"] = r["achieved"] / r["peak"] if r["peak"] else None
                out["taylor_update_share_of_step"] = acc["ms_total"] / ms
        if prec == "mixed":
            Q.qm_hpsi_prepare(g.handle, 0, None)
        del psi, beta, work
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    g.close()
    torch.cuda.empty_cache()
    return out


def run_gw(args, Q, S, dev):
    """GW plane-wave matrix elements on the 64-atom cell (72^3): k and k+q two points of its shifted
    set, 32 states at k+q times 64 at k (2048 pairs), E_eps a quarter of the wavefunction cutoff;
    both precisions, CUDA events around the calls."""
    import numpy as np
    import torch
    cell = S.config2()
    k, kq = cell.kpts[0], cell.kpts[1]
    g = Q.GSpace(cell.lattice, [kq, k], cell.ecut_ha, cell.grid)
    ge = Q.GSpace(cell.lattice, [kq - k], 0.25 * cell.ecut_ha, cell.grid)
    nl, nr = 32, 64
    out = {"workload": "si64_cubic_72^3_%dx%d_pairs_eps_quarter" % (nl, nr), "pairs": nl * nr,
           "npw_eps": ge.npw[0], "unit": "pairs/s"}
    stream = torch.cuda.current_stream()
    for prec, steps in (("mixed", 5), ("fp64", 2)):
        cdt = torch.complex64 if prec == "mixed" else torch.complex128
        pl = torch.from_numpy(S.psi_random(cell.seed, nl, g.npw[0], stream=1)).to(cdt).to(dev)
        pr = torch.from_numpy(S.psi_random(cell.seed, nr, g.npw[1], stream=0)).to(cdt).to(dev)
        M = torch.empty((nl * nr, ge.npw[0]), dtype=cdt, device=dev)
        Q.qm_gw_mel(g.handle, 0, 1, pl, pr, ge.handle, 0, ge.npw[0], M=M, prec=prec, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            Q.qm_gw_mel(g.handle, 0, 1, pl, pr, ge.handle, 0, ge.npw[0], M=M, prec=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"value": nl * nr / (ms * 1e-3), "ms_per_call": ms, "steps": steps}
        # the pair phase reads two real-space boxes per pair: those bytes over the whole call's time
        # (the states' transforms to real space and the gathers included in the time)
        nbytes = nl * nr * 2.0 * (cell.grid[0] * cell.grid[1] * cell.grid[2]) * (8 if prec == "mixed" else 16)
        pk = load_peaks()[0].get("hbm_gbs")
        out[prec]["pair_reads"] = {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": pk, "unit": "GB/s",
                                   "frac": nbytes / (ms * 1e-3) / 1e9 / pk if pk else None,
                                   "bytes_per_call": nbytes}
        del pl, pr, M
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    ge.close()
    g.close()
    torch.cuda.empty_cache()
    return out


def run_scf(args, Q, S, dev):
    """Kohn-Sham self-consistency (qm_scf) on the 8-atom cubic cell (15 Ry, the grid rule's grid,
    the shifted 2x2x2 k-points, 8 bands, the lowest band occupied: 2 electrons), from random states
    and the uniform density to a density residual of 1e-8 electrons; wall time of the call."""
    import torch
    cell = S.cubic_si8(15.0, nbnd=8, kpts=S.config2().kpts)
    g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, None)
    grid = g.grid
    vion = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, grid)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    ld = max(g.npw)   # one row stride for every k-point
    betas = []
    for ik in range(len(cell.kpts)):
        _, _, kpg = g.indices(ik)
        b = torch.zeros((cell.nproj, ld), dtype=torch.complex128)
        b[:, :g.npw[ik]] = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega))
        betas.append(b.to(dev))
    w = [1.0 / len(cell.kpts)] * len(cell.kpts)
    out = {"workload": "si8_cubic_15Ry_%dx%dx%d_4k_8b_2e" % tuple(grid), "npw": g.npw, "tol_electrons": 1e-8}
    for prec in ("fp64", "mixed"):
        psis = []
        for ik in range(len(cell.kpts)):
            p = torch.zeros((cell.nbnd, ld), dtype=torch.complex128)
            p[:, :g.npw[ik]] = torch.from_numpy(S.psi_random(cell.seed, cell.nbnd, g.npw[ik], stream=ik))
            psis.append(p.to(dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eig, rho, v, info = Q.qm_scf(g.handle, 2, w, psis, vion, betas, D, tol=1e-8, prec=prec)
        torch.cuda.synchronize()
        out[prec] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                     "converged": info["converged"], "band_applies": info["band_applies"],
                     "lowest_eigenvalue_ha": float(eig[:, 0].min())}
        if prec == "mixed":
            out["max_eig_diff_vs_fp64_ha"] = float(abs(eig - out["fp64"].pop("_eig")).max())
        else:
            out[prec]["_eig"] = eig
    out["fp64_over_mixed_seconds"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    g.close()
    return out


def run_ours(args):
    import torch

    import paper_2308_07277_gb300 as Q
    import qm_synth as S
    from paper_2308_07277_gb300 import _lib

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = _lib.load()
    peaks, _ = load_peaks()

    def hpsi_forms(cell, head_clocks, e2e_mixed):
        g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
        v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
        D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
        res, wls = {}, {}
        for prec in ("mixed", "fp64"):
            wl = Workload(S, g, cell, rank, prec, dev)
            if prec == "mixed":
                # the projectors split on every call (qm_hpsi alone) ...
                res["mixed_per_call"] = measure_hpsi(max(3, args.steps // 3), args.warmup, Q, lib, g, cell, wl, v, D,
                                                     world, dev, peaks, sample_clocks=False, with_e2e=False)
                # ... and prepared once per k-point (qm_hpsi_prepare: the projectors are fixed for a
                # k-point, as in every Davidson iteration); setup time reported, not timed per step
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for ik in range(len(cell.kpts)):
                    Q.qm_hpsi_prepare(g.handle, ik, wl.beta[ik])
                torch.cuda.synchronize()
                prep_s = time.perf_counter() - t0
            # the FP64 form runs ~60x slower: fewer timed steps (at least 2)
            steps = args.steps if prec == "mixed" else max(2, args.steps // 10)
            warm = args.warmup if prec == "mixed" else 1
            res[prec] = measure_hpsi(steps, warm, Q, lib, g, cell, wl, v, D, world, dev, peaks,
                                     sample_clocks=head_clocks and prec == "mixed",
                                     with_e2e=e2e_mixed and prec == "mixed")
            res[prec]["steps"] = steps
            if prec == "mixed" and head_clocks:
                res["fft_path"] = measure_fft_path(steps, warm, Q, g, cell, wl, v, res[prec]["kernels"],
                                                   res[prec]["ms_per_step"], peaks)
            if prec == "mixed":
                res[prec]["prepare_seconds"] = prep_s
                for ik in range(len(cell.kpts)):
                    Q.qm_hpsi_prepare(g.handle, ik, None)
            wls[prec] = wl
        return g, v, D, res, wls

    # headline: the 255-atom cell
    cell = S.config5()
    g, v, D, forms, wls = hpsi_forms(cell, True, True)
    npw5 = list(g.npw)
    del wls
    g.close()
    torch.cuda.empty_cache()
    # the 64-atom cell: both forms, and the Davidson solves on it
    cell2 = S.config2()
    g2, v2, D2, forms2, wl2 = hpsi_forms(cell2, False, False)
    dav = run_davidson(args, Q, lib, g2, cell2, wl2["fp64"], v2, D2) if args.davidson else None
    del wl2
    g2.close()
    torch.cuda.empty_cache()
    batched = run_batched(args, Q, S, dev) if args.batched else None
    tddft = run_tddft(args, Q, S, dev) if args.tddft else None
    gw = run_gw(args, Q, S, dev) if args.gw else None
    scf = run_scf(args, Q, S, dev) if args.scf else None
    large = run_large_cells(args, Q, S, dev) if args.large else None
    theta, tinfo = train_network(Q, S, dev) if (args.davidson_large or args.davidson_255) else (None, None)
    dav255 = run_davidson_255(args, Q, S, dev, theta) if args.davidson_255 else None
    dav_large = run_davidson_large(args, Q, S, dev, theta) if args.davidson_large else None
    if rank == 0:
        head = forms["mixed"]
        keep = ("value", "ms_per_step", "steps", "roofline", "roofline_other", "kernels", "gpu_launches")
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3", "data": "synthetic",
                "config": {"workload": WORKLOAD,
                           "precision": "mixed (FP32 FFT path, BF16x3-split tensor-core nonlocal GEMMs)",
                           "projectors": "prepared once per k-point (qm_hpsi_prepare, %.3f s, outside the timed "
                                         "steps); per-call splitting under forms.mixed_per_call" % head["prepare_seconds"],
                           "band_applies_per_step": cell.nbnd * len(cell.kpts), "npw": npw5,
                           "nproj": cell.nproj, "grid": list(cell.grid), "l2": head["l2"]},
                "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "kernels": head["kernels"],
                "roofline": head["roofline"], "roofline_other": head["roofline_other"],
                "fft_path": forms.get("fft_path"),
                "clocks": head["clocks"],
                "forms": {"fp64": {k: forms["fp64"][k] for k in keep},
                          "mixed_per_call": {k: forms["mixed_per_call"][k] for k in keep if k in forms["mixed_per_call"]},
                          "mixed_over_fp64": head["value"] / forms["fp64"]["value"]},
                "config2": {"workload": WORKLOAD2, "band_applies_per_step": cell2.nbnd * len(cell2.kpts),
                            "mixed": {k: forms2["mixed"][k] for k in keep},
                            "mixed_per_call": {k: forms2["mixed_per_call"][k] for k in keep if k in forms2["mixed_per_call"]},
                            "fp64": {k: forms2["fp64"][k] for k in keep},
                            "mixed_over_fp64": forms2["mixed"]["value"] / forms2["fp64"]["value"]},
                "davidson": dav,
                "davidson_255_atoms": dav255,
                "learned_training": tinfo,
                "batched": batched,
                "tddft": tddft,
                "gw_matrix_elements": gw,
                "scf": scf,
                "large_cells": large,
                "davidson_216_atoms_learned": dav_large,
                "cpu_baseline": oracle_sample("config5", args.cpu_baseline_bands)}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """Only the kernels a profiler should see: the precision form's H psi steps on one cell (all
    k-points or the first --profile-k), projectors prepared, or replays of the batched form."""
    import torch

    import paper_2308_07277_gb300 as Q
    import qm_synth as S
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.profile_batched:
        prec = args.profile_batched
        cells = S.config3_cells(lambda c: product_grid(Q, c))
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        gss, jobs = [], []
        for cell in cells:
            g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
            gss.append(g)
            v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid, cell.depth, cell.width,
                                                ortho_period=cell.ortho_period)).to(dev)
            D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
            for ik in range(len(cell.kpts)):
                _, _, kpg = g.indices(ik)
                psi = torch.from_numpy(S.psi_random(cell.seed, cell.nbnd, g.npw[ik], stream=ik)).to(cdt).to(dev)
                beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega, cell.rc)).to(cdt).to(dev)
                jobs.append({"g": g.handle, "ik": ik, "psi": psi, "vloc": v, "beta": beta, "D": D,
                             "out": torch.empty_like(psi)})
        shape = dict(ctas_per_sm=3, item_points=8192, group_mb=-1) if prec == "mixed" else \
            dict(ctas_per_sm=1, item_points=8192, group_mb=-1)
        b = Q.Batch(jobs, prec=prec, **shape)
        for _ in range(args.warmup + args.steps):
            b.run()
        b.check()
        torch.cuda.synchronize()
        print(json.dumps({"profile": "batched", "prec": prec, "replays": args.warmup + args.steps, **b.info()}))
        return
    if args.profile == "gw":
        # the GW matrix elements of the benchmark's workload (64-atom cell, 32 x 64 pairs), one
        # call per step in the --profile-prec precision
        cell = S.config2()
        k, kq = cell.kpts[0], cell.kpts[1]
        g = Q.GSpace(cell.lattice, [kq, k], cell.ecut_ha, cell.grid)
        ge = Q.GSpace(cell.lattice, [kq - k], 0.25 * cell.ecut_ha, cell.grid)
        cdt = torch.complex64 if args.profile_prec == "mixed" else torch.complex128
        pl = torch.from_numpy(S.psi_random(cell.seed, 32, g.npw[0], stream=1)).to(cdt).to(dev)
        pr = torch.from_numpy(S.psi_random(cell.seed, 64, g.npw[1], stream=0)).to(cdt).to(dev)
        M = torch.empty((32 * 64, ge.npw[0]), dtype=cdt, device=dev)
        for _ in range(args.warmup + args.steps):
            Q.qm_gw_mel(g.handle, 0, 1, pl, pr, ge.handle, 0, ge.npw[0], M=M, prec=args.profile_prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "gw", "precision": args.profile_prec, "steps": args.warmup + args.steps}))
        ge.close()
        g.close()
        return
    cell = getattr(S, args.profile)()
    nk = args.profile_k or len(cell.kpts)
    prec = args.profile_prec
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    g = Q.GSpace(cell.lattice, cell.kpts[:nk], cell.ecut_ha, cell.grid)
    v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    psi, beta, out = [], [], []
    for ik in range(nk):
        _, _, kpg = g.indices(ik)
        psi.append(torch.from_numpy(S.psi_random(cell.seed, cell.nbnd, g.npw[ik], stream=ik)).to(cdt).to(dev))
        beta.append(torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(cdt).to(dev))
        out.append(torch.empty_like(psi[-1]))
        if prec == "mixed":
            Q.qm_hpsi_prepare(g.handle, ik, beta[-1])
    for _ in range(args.warmup + args.steps):
        for ik in range(nk):
            Q.qm_hpsi(g.handle, ik, psi[ik], v, beta[ik], D, out=out[ik], prec=prec)
    torch.cuda.synchronize()
    print(json.dumps({"profile": cell.name, "precision": prec, "k_points": nk, "steps": args.warmup + args.steps}))
    g.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile or args.profile_batched:
        run_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
