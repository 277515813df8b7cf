"""H-psi throughput benchmark on the 64-atom Si-like cubic cell (a = 20.52 bohr, 25 Ry,
FFT grid 72^3, 4 shifted k-points, 160 bands, 256 projectors, 18,232 plane waves per k).

One step = H psi applied to every band at every k-point (640 band-applies) through the
C ABI (qm_hpsi).  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|mixed] [--impl reference]

--impl reference times the FP64 CPU oracle (numpy, one thread) on a bounded sample of
the same workload: it is a deliberately slow baseline, not a competitor.
Multi-GPU (torchrun, one process per GPU): every rank processes its own copy of the cell
(independent problems, no collective on the data path), "scaling": "weak".
"""
from __future__ import annotations

import argparse
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
WORKLOAD = "si64_cubic_72^3_4k_160b"

# FP64 / FP32 ALU peaks derived from SM count x per-SM FMA units x max clock:
#   FP64: nominal 1.25 TFLOP/s over 152 SMs at 2.07 GHz = 4 flop/clk/SM (2 DFMA/clk/SM)
#   FP32: 128 FMA/clk/SM
N_SM = 152
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-sample-bands", type=int, default=48)
    ap.add_argument("--davidson", type=int, default=1, help="also time block Davidson to tol (0: skip)")
    ap.add_argument("--davidson-tol", type=float, default=1e-8)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        mine = [r for r in rows if self.bus and self.bus[-12:] in r[0].lower()] or rows
        sm = sorted(float(r[1]) for r in mine if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in mine if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in mine for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(mine)}


# ------------------------------------------------------------------ oracle (CPU) leg
def oracle_sample(nbands):
    """Time the FP64 oracle (numpy, one BLAS thread) on nbands bands of k-point 0."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import qm_synth as S
from oracle import gspace as OG, hamiltonian as OH
c = S.config2()
gs = OG.gsphere(c.lattice, c.grid, c.ecut_ha, c.kpts[0])
v = S.vloc_on_grid(c.lattice, c.tau, c.grid)
beta = S.beta_of_q(gs['q'], c.tau, c.omega)
D = S.dvals(c.nat)
psi = S.psi_random(1, {nbands}, len(gs['idx']))
OH.hpsi_fft(psi[:1], gs, v, beta, D)
t = time.perf_counter()
OH.hpsi_fft(psi, gs, v, beta, D)
dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt, "bands": {nbands}}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode:
        raise RuntimeError("oracle leg failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["bands"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['bands']} bands of k-point 0 (of 640 band-applies per step), FP64 numpy "
                      f"full-box FFT + nonlocal, 1 thread, {d['seconds']:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    nb = max(1, args.cpu_sample_bands // 8)
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(nb)
        if i >= args.warmup:
            vals.append(r["value"])
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 640 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64", "sample_bands_per_step": nb},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{nb} bands of k-point 0 per step, FP64 numpy oracle, 1 thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU leg
def fft_flops_per_plane_launch(grid, nrow):
    """Algorithmic flops of one k_plane CTA (one band, one yz plane), 5 L log2 L per FFT."""
    n1, n2, n3 = grid
    f = lambda L: 5.0 * L * math.log2(L)
    return 2.0 * (nrow * f(n2) + n2 * f(n3)) + 2.0 * n2 * n3


def read_prof(lib):
    import ctypes
    fam = {}
    for f in range(9):
        t = ctypes.c_double()
        c = ctypes.c_longlong()
        lib.qm_prof_read(f, ctypes.byref(t), ctypes.byref(c))
        if c.value:
            fam[lib.qm_prof_name(f).decode()] = {"ms_total": t.value, "launches": c.value}
    return fam


def run_davidson(args, Q, lib, g, cell, psi_host, v, beta, D, nk, nb):
    """Block Davidson to a residual of args.davidson_tol at every k-point (FP64 H psi),
    from the seeded random start; wall time of the qm_davidson calls."""
    import torch
    if args.prec != "fp64":
        return {"skipped": "the Davidson leg runs the FP64 form"}
    per_k = []
    lib.qm_prof_enable(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ik in range(nk):
        p = psi_host[ik].to(torch.complex128).cuda()
        eig, info = Q.qm_davidson(g.handle, ik, p, v, beta[ik].to(torch.complex128), D, tol=args.davidson_tol,
                                  max_iter=300, raise_not_converged=False)
        per_k.append({"iterations": info["iterations"], "band_applies": info["band_applies"],
                      "max_residual": info["max_residual"], "converged": info["converged"],
                      "seconds": info["seconds"], "eig_min": float(eig[0]), "eig_max": float(eig[-1])})
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    fam = read_prof(lib)
    lib.qm_prof_enable(0)
    return {"precision": "fp64", "tol_ha": args.davidson_tol, "seconds_total": total, "nbnd": nb,
            "per_k": per_k, "kernels": fam}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2308_07277_gb300 as Q
    import qm_synth as S
    from paper_2308_07277_gb300 import _lib

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = _lib.load()
    cell = S.config2()
    prec = args.prec
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    nk, nb, nproj = len(cell.kpts), cell.nbnd, cell.nproj
    v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).to(dev)
    D = torch.from_numpy(S.dvals(cell.nat)).to(dev)
    psi, beta, out, psi_host, out_host, nrow = [], [], [], [], [], []
    for ik in range(nk):
        idx, _, kpg = g.indices(ik)
        nrow.append(len(np.unique(idx // (cell.grid[0] * cell.grid[1]))))   # yz-plane rows holding sticks
        npw = g.npw[ik]
        p = S.psi_random(cell.seed + rank, nb, npw, stream=ik)
        psi_host.append(torch.from_numpy(p).to(cdt).pin_memory())
        psi.append(psi_host[-1].to(dev))
        beta.append(torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(cdt).to(dev))
        out.append(torch.empty_like(psi[-1]))
        out_host.append(torch.empty_like(psi_host[-1]).pin_memory())
    stream = torch.cuda.current_stream()

    def step():
        for ik in range(nk):
            Q.qm_hpsi(g.handle, ik, psi[ik], v, beta[ik], D, out=out[ik], prec=prec, stream=stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", ""))
    clocks.start()
    time.sleep(0.3)
    lib.qm_prof_enable(1)
    n0 = lib.qm_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    launches = int(lib.qm_launch_count() - n0)
    ms = e0.elapsed_time(e1) / args.steps
    fam = {}
    import ctypes
    for f in range(9):
        t = ctypes.c_double()
        c = ctypes.c_longlong()
        lib.qm_prof_read(f, ctypes.byref(t), ctypes.byref(c))
        if c.value:
            fam[lib.qm_prof_name(f).decode()] = {"ms_total": t.value, "launches": c.value}
    lib.qm_prof_enable(0)
    clk = clocks.stop()

    # end to end: pinned host psi -> device, H psi, device -> pinned host, every step
    for _ in range(2):
        for ik in range(nk):
            psi[ik].copy_(psi_host[ik], non_blocking=True)
        step()
        for ik in range(nk):
            out_host[ik].copy_(out[ik], non_blocking=True)
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    esteps = max(3, args.steps // 3)
    for _ in range(esteps):
        for ik in range(nk):
            psi[ik].copy_(psi_host[ik], non_blocking=True)
        step()
        for ik in range(nk):
            out_host[ik].copy_(out[ik], non_blocking=True)
    e3.record(stream)
    barrier()
    ems = e2.elapsed_time(e3) / esteps
    h2d = sum(t.numel() * t.element_size() for t in psi_host)
    d2h = sum(t.numel() * t.element_size() for t in out_host)

    dav = run_davidson(args, Q, lib, g, cell, psi_host, v, beta, D, nk, nb) if args.davidson else None

    if world > 1:
        t = torch.tensor([ms, ems], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ems = float(t[0]), float(t[1])
    band_applies = nb * nk * world
    value = band_applies / (ms * 1e-3)

    line = None
    if rank == 0:
        peaks, peak_src = load_peaks()
        dom = max(fam.items(), key=lambda kv: kv[1]["ms_total"]) if fam else None
        roof = None
        if dom is not None:
            name, d = dom
            avg_ms = d["ms_total"] / d["launches"]
            smax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
            fl_pk = (FP64_FLOP_PER_CLK_SM if prec == "fp64" else FP32_FLOP_PER_CLK_SM) * N_SM * smax / 1e12
            if name == "k_plane":
                # algorithmic flops of one step's planes (nb x N1 per k), spread over its launches
                per_step = d["launches"] / args.steps
                fl = sum(nb * cell.grid[0] * fft_flops_per_plane_launch(cell.grid, nrow[ik]) for ik in range(nk))
                fl /= per_step
                roof = {"bound": "alu", "achieved": fl / (avg_ms * 1e-3) / 1e12, "peak": fl_pk, "unit": "TFLOP/s"}
            elif name in ("k_gemm_tn", "k_gemm_cn"):
                # nonlocal GEMMs: 8 flops per complex multiply-add, nproj x nb x npw per k
                per_step = d["launches"] / args.steps
                fl = 8.0 * nproj * nb * g.npw[0] * nk / per_step
                roof = {"bound": "alu", "achieved": fl / (avg_ms * 1e-3) / 1e12, "peak": fl_pk, "unit": "TFLOP/s"}
            else:
                roof = {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s"}
            roof["kernel"] = name
            roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("achieved") else None
            roof["traffic"] = None
            roof["peak_source"] = "derived: %d SMs x %d flop/clk/SM x %.0f MHz (%s clock)" % (
                N_SM, FP64_FLOP_PER_CLK_SM if prec == "fp64" else FP32_FLOP_PER_CLK_SM, smax / 1e6, peak_src)
            roof["avg_launch_ms"] = avg_ms
        cpu = oracle_sample(args.cpu_sample_bands) if world == 1 or rank == 0 else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": prec, "band_applies_per_step": nb * nk,
                           "npw": g.npw[0], "nproj": nproj, "grid": list(cell.grid),
                           "l2": "inputs larger than L2: psi %.0f MB + beta %.0f MB per step" % (
                               h2d / 1e6, sum(b.numel() * b.element_size() for b in beta) / 1e6)},
                "e2e": {"value": band_applies / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": ems},
                "gpu_launches": launches,
                "kernels": fam,
                "roofline": roof,
                "cpu_baseline": cpu,
                "clocks": clk,
                "davidson": dav}
        print(json.dumps(line))
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
