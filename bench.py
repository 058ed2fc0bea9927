#!/usr/bin/env python
"""Throughput of one SevenNet energy + force + virial evaluation on a GB300.

A step is one full evaluation (cell-list neighbour build, five interaction
blocks forward, the hand-written adjoint, forces and virial) of the
24,000-atom SiO2 cell with the 5-layer 128x0e+64x1e+32x2e model, inputs
resident in HBM.  metric: atom-steps/s (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)
  python bench.py --workload sio2_3000 --precision fp32 --md-steps 100
  python bench.py --workload si3n4_112000 --md-steps 1000
      NVE velocity-Verlet MD through sevennet_md_step (1 fs, Maxwell-Boltzmann
      velocities at 3000 K); a step is one evaluation with its neighbour rebuild
      plus the position and velocity update; reports atom-steps/s and the drift
      of the total energy.

Under torchrun (N > 1) every rank evaluates its own replica (the evaluation
does not shard: replicas only); value = all ranks' atom-steps / the slowest
rank's time.
"""

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
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (E+F+virial)"
UNIT = "atom-steps/s"
WORKLOAD = "sio2_24000"

# non-zero real Clebsch-Gordan coefficients of each coupling (l1, l2, l3)
CG_NNZ = {(0, 0, 0): 1, (0, 1, 1): 3, (0, 2, 2): 5, (1, 0, 1): 3, (1, 1, 0): 3, (1, 1, 1): 6,
          (1, 1, 2): 11, (1, 2, 1): 11, (1, 2, 2): 16, (2, 0, 2): 5, (2, 1, 1): 11, (2, 1, 2): 16,
          (2, 2, 0): 5, (2, 2, 1): 16, (2, 2, 2): 25}


def block_paths(spec, t):
    lmax = len(spec.mul) - 1
    first, last = t == 0, t == spec.n_layers - 1
    in_mul = {0: spec.mul[0]} if first else {l: spec.mul[l] for l in range(lmax + 1)}
    out = []
    for l1 in sorted(in_mul):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if last and l3 != 0:
                    continue
                out.append((l1, l2, l3, in_mul[l1]))
    return out


def conv_flops_per_edge(spec, t, adjoint, tensor_core):
    """Algorithmic FLOPs of the fused convolution kernel per edge for block t,
    split into (FFMA work, tensor-core work).  With tensor_core, the MLP matrix
    products with H-wide inputs (H x H and H x W) run on tensor cores.  The
    adjoint of an evaluation runs over unordered pairs of edges: the radial MLP
    (recompute and input gradient) and the G matrices once per pair, the tensor
    product once per direction, so per edge the former count half."""
    H, NB = spec.mlp_hidden, spec.n_basis
    paths = block_paths(spec, t)
    W = sum(p[3] for p in paths)
    first = 2 * NB * H                                         # basis -> hidden, FFMA always
    mm = 2 * (H * H + H * W)                                   # hidden -> hidden -> W
    g = sum(2 * CG_NNZ[p[:3]] for p in paths)                 # G matrices
    if not adjoint:
        tp = sum(2 * mu * ((2 * l1 + 1) * (2 * l3 + 1) + (2 * l3 + 1)) for l1, l2, l3, mu in paths)
        mlp_alu, mlp_tc = (first, mm) if tensor_core else (first + mm, 0)
        return mlp_alu + g + tp, mlp_tc
    tp = sum(2 * mu * ((2 * l1 + 1) * (2 * l3 + 1) + 2 * (2 * l1 + 1) + CG_NNZ[(l1, l2, l3)])
             for l1, l2, l3, mu in paths)
    # forward recompute + input gradient of the MLP, and the G matrices, once per pair
    mlp_alu, mlp_tc = (first, mm) if tensor_core else (first + mm, 0)
    return mlp_alu + g // 2 + tp, mlp_tc


def fp32_alu_peak_tflops(n_sm, clock_mhz):
    """FFMA peak from unit counts: SMs x 128 FP32 lanes x 2 FLOP x clock."""
    return n_sm * 128 * 2 * clock_mhz * 1e6 / 1e12


def measure_alu_peak(sn, device, seconds=1.5):
    """FP32 FMA throughput measured by the library's microbenchmark
    (sevennet_fp32_peak: register-resident independent FMA chains), scalar and
    packed (f32x2) forms alternated for `seconds` with the SM clock sampled."""
    clk = ClockSampler(device)
    clk.start()
    time.sleep(0.3)
    res = {False: [], True: []}
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end:
        for packed in (False, True):
            res[packed].append(sn.SevenNet.fp32_peak(device, packed, 200000)[0])
    clk.stop()
    c = clk.summary()
    out = {"ffma_tflops": max(res[False]), "ffma2_tflops": max(res[True]), "launches": len(res[False]) * 4,
           "clocks": c, "how": "sevennet_fp32_peak: 4 CTAs x 256 threads per SM, 16 independent FMA chains "
                               "per thread, 200,000 iterations, best launch"}
    out["peak_tflops"] = max(out["ffma_tflops"], out["ffma2_tflops"])
    if c.get("sm_mhz"):
        out["flop_per_sm_cycle"] = out["peak_tflops"] * 1e12 / (c["sm_mhz"] * 1e6) / sn_count_sms(device)
    return out


def sn_count_sms(device):
    import torch
    return torch.cuda.get_device_properties(device).multi_processor_count


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(steps=None, seconds=12.0):
    """Time the FP64 CPU oracle on the bounded sample (cpu_baseline leg)."""
    import torch
    import oracle
    from synth import make_workload, normal_weights
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    torch.set_num_threads(cores)
    s, spec = make_workload("sio2_192_l2")
    w = normal_weights(oracle.n_params(spec))
    oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)     # CG tables, warm caches
    n_done, t0 = 0, time.perf_counter()
    res = None
    while True:
        res = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
        n_done += 1
        el = time.perf_counter() - t0
        if (steps is not None and n_done >= steps) or (steps is None and el >= seconds):
            break
    return dict(value=s.n_atoms * n_done / el, unit=UNIT, cores=torch.get_num_threads(), kind="oracle",
                sample=f"{n_done} E+F+virial evaluations of a 192-atom SiO2 cell (2.2 g/cm3, same "
                       f"5-layer model) by the FP64 CPU oracle"), (s, spec, w, res)


def traffic_for(kernel):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ent = json.load(open(path)).get(kernel)
        h = hashlib.sha256()
        for f in ent["source_files"]:
            h.update(open(os.path.join(ROOT, "paper_2402_03789_gb300", "csrc", f), "rb").read())
        if h.hexdigest()[:16] == ent["source_sha"]:
            return ent["bytes_per_launch_full_workload"]
    except Exception:
        pass
    return None


def serving_run(sn, model, precision, n_requests=512, rate_hz=200.0, budget_gb=8.0, n_streams=4,
                max_batch=32):
    """Replay the Poisson request stream through the continuous-batching server.

    Requests are submitted at their arrival times; latency = completion - arrival
    on the server clock.  Returns p50/p99 latency, throughput and batching stats.
    At an offered rate above the server's capacity the queue fills and the
    throughput is the server's own (saturated).
    """
    from synth import serving_trace
    trace = serving_trace(n_requests, rate_hz, seed=6)
    srv = sn.Server(model, hbm_budget_bytes=int(budget_gb * (1 << 30)), n_streams=n_streams,
                    max_batch_structs=max_batch, precision=precision)
    # warm the server's buffers with a few requests (not counted)
    warm = [srv.submit(st.pos, st.cell, st.species) for _, st in trace[:8]]
    for t in warm:
        while srv.poll(t) is None:
            time.sleep(0.0005)
    t0 = srv.now()
    pending, done = {}, {}
    i = 0
    while i < len(trace) or pending:
        now = srv.now() - t0
        while i < len(trace) and trace[i][0] <= now:
            st = trace[i][1]
            pending[srv.submit(st.pos, st.cell, st.species)] = (i, st.n_atoms)
            i += 1
        for tk in list(pending):
            r = srv.poll(tk)
            if r is not None:
                done[tk] = (r, pending.pop(tk)[1])
        if i < len(trace):
            time.sleep(max(0.0, min(0.0005, trace[i][0] - (srv.now() - t0))))
        else:
            time.sleep(0.0002)
    srv.close()
    lat = sorted((r["done_s"] - r["submit_s"]) * 1e3 for r, _ in done.values())
    first = min(r["submit_s"] for r, _ in done.values())
    last = max(r["done_s"] for r, _ in done.values())
    atoms = sum(n for _, n in done.values())
    bsz = [r["batch_structs"] for r, _ in done.values()]
    return {"requests": len(done), "rate_hz": rate_hz, "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "max_ms": lat[-1],
            "atom_steps_per_s": atoms / (last - first), "mean_batch_structs": sum(bsz) / len(bsz),
            "streams": n_streams, "hbm_budget_gb": budget_gb, "precision": precision,
            "trace": f"{n_requests} cells of 16-2000 atoms (log-uniform), Si/N/O, 2.2-3.1 g/cm3, "
                     f"Poisson arrivals at {rate_hz:.0f}/s"}


# initial-velocity seeds of the MD workloads (3000 K)
MD_VEL_SEED = {"sio2_3000": 3, "si3n4_112000": 8}


def md_leg(sn, model, workload, precision, steps, warmup=3, device=0):
    """NVE MD of one workload through sevennet_md_step (1 fs, Maxwell-Boltzmann
    velocities at 3000 K): atom-steps/s by the host clock around one md_step call
    of `steps` steps (one host synchronisation per call), and the drift of the
    total energy."""
    import numpy as np
    import torch
    from synth import make_workload, maxwell_boltzmann
    from synth.configs import MASSES_AMU
    s, _ = make_workload(workload)
    masses = np.asarray(MASSES_AMU)
    vel = maxwell_boltzmann(masses[s.species], 3000.0, seed=MD_VEL_SEED.get(workload, 3))
    md = sn.MD(model, s.pos, vel, s.species, masses, s.cell, precision)
    md.step(warmup, 1.0)
    clk = ClockSampler(device)
    torch.cuda.synchronize()
    clk.start()
    t0 = time.perf_counter()
    ep, ek = md.step(steps, 1.0)
    wall = time.perf_counter() - t0
    clk.stop()
    md.close()
    etot = ep + ek
    n = s.n_atoms
    return {"workload": workload, "n_atoms": n, "precision": precision, "steps": steps, "warmup": warmup,
            "dt_fs": 1.0, "ensemble": "NVE", "T_init_K": 3000.0,
            "value": n * steps / wall, "unit": UNIT, "ms_per_step": wall * 1e3 / steps,
            "etot_drift_eV_per_atom": float((etot[-1] - etot[0]) / n),
            "etot_max_dev_eV_per_atom": float(np.max(np.abs(etot - etot[0])) / n),
            "timing": "host wall clock around one sevennet_md_step call", "clocks": clk.summary()}


def md_run(args, world, rank, dev, sn, model, s):
    """NVE MD through the C ABI: atom-steps/s and total-energy drift."""
    import numpy as np
    import torch
    from synth import maxwell_boltzmann
    from synth.configs import MASSES_AMU
    masses = np.asarray(MASSES_AMU)
    vel = maxwell_boltzmann(masses[s.species], 3000.0, seed=MD_VEL_SEED.get(args.workload, 3))
    md = sn.MD(model, s.pos, vel, s.species, masses, s.cell, args.precision)
    if args.skin > 0:
        md.set_skin(args.skin)
    if args.nvt > 0:
        md.set_nose_hoover(args.nvt, args.tau)
    md.step(args.warmup, 1.0)
    builds0, _ = md.stats()
    clk = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize(dev)
    clk.start()
    t0 = time.perf_counter()
    ep, ek = md.step(args.md_steps, 1.0)
    torch.cuda.synchronize(dev)
    wall = max_over_ranks(time.perf_counter() - t0, world, dev)
    clk.stop()
    builds, _ = md.stats()
    etot = ep + ek
    n = s.n_atoms
    ensemble = {"ensemble": "NVE"}
    if args.nvt > 0:
        xi, eta = md.nose_hoover()
        kb = 8.617333262e-5
        nf = 3 * n - 3
        q = nf * kb * args.nvt * args.tau ** 2
        ext = etot[-1] + 0.5 * q * xi * xi + nf * kb * args.nvt * eta
        ensemble = {"ensemble": "NVT Nose-Hoover", "T0_K": args.nvt, "tau_fs": args.tau,
                    "T_final_K": float(2 * ek[-1] / (nf * kb)), "extended_energy_final_eV": float(ext)}
    line = {"metric": "atom-steps/s (MD: neighbour list + E+F+virial + Verlet update)",
            "value": world * n * args.md_steps / wall, "unit": UNIT, "n_gpus": world, "steps": args.md_steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.md_steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_atoms": n, "precision": args.precision, "dt_fs": 1.0,
                       "T_init_K": 3000.0, "skin_A": args.skin, "timing": "host wall clock around sevennet_md_step",
                       "parallelism": f"replicas x{world}"} | ensemble,
            "md": {"epot0_eV_per_atom": float(ep[0] / n), "ekin0_eV_per_atom": float(ek[0] / n),
                   "etot_drift_eV_per_atom": float((etot[-1] - etot[0]) / n),
                   "etot_max_dev_eV_per_atom": float(np.max(np.abs(etot - etot[0])) / n),
                   "finite": bool(np.all(np.isfinite(etot))),
                   "neighbour_builds_in_timed_steps": int(builds - builds0)},
            "clocks": clk.summary()}
    md.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def melt_quench_run(args, world, rank, dev, sn, model, s):
    """The melt-quench protocol of Sec. 5.2 under Nose-Hoover NVT, every
    duration multiplied by args.melt_quench: hold at 5000 K for 10 ps, hold at
    3000 K for 20 ps, quench to 2000 K at -33 K/ps (30.3 ps); dt = 1 fs.
    atom-steps/s over the whole schedule and the temperature at the end of each
    segment."""
    import numpy as np
    import torch
    from synth import maxwell_boltzmann
    from synth.configs import MASSES_AMU
    masses = np.asarray(MASSES_AMU)
    f = args.melt_quench
    segs = [("hold", 5000.0, max(1, int(round(10000 * f)))),
            ("hold", 3000.0, max(1, int(round(20000 * f)))),
            ("ramp", 3000.0, 2000.0, max(1, int(round(1000.0 / 33.0 * 1000 * f))))]
    vel = maxwell_boltzmann(masses[s.species], 5000.0, seed=MD_VEL_SEED.get(args.workload, 3))
    md = sn.MD(model, s.pos, vel, s.species, masses, s.cell, args.precision)
    if args.skin > 0:
        md.set_skin(args.skin)
    md.set_nose_hoover(5000.0, args.tau)
    md.step(args.warmup, 1.0)
    clk = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize(dev)
    clk.start()
    t0 = time.perf_counter()
    ep, ek = md.run_schedule(segs, 1.0, args.tau)
    torch.cuda.synchronize(dev)
    wall = max_over_ranks(time.perf_counter() - t0, world, dev)
    clk.stop()
    n, steps = s.n_atoms, len(ep)
    kb, nf = 8.617333262e-5, 3 * s.n_atoms - 3
    ends = np.cumsum([sg[-1] for sg in segs]) - 1
    line = {"metric": "atom-steps/s (NVT melt-quench schedule of Sec. 5.2, time-scaled)",
            "value": world * n * steps / wall, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_atoms": n, "precision": args.precision, "dt_fs": 1.0,
                       "time_scale": f, "schedule": [list(sg) for sg in segs], "tau_fs": args.tau,
                       "skin_A": args.skin, "timing": "host wall clock around the schedule",
                       "parallelism": f"replicas x{world}"},
            "melt_quench": {"T_end_of_segment_K": [float(2 * ek[i] / (nf * kb)) for i in ends],
                            "epot_final_eV_per_atom": float(ep[-1] / n),
                            "finite": bool(np.all(np.isfinite(ep + ek)))},
            "clocks": clk.summary()}
    md.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def paper_sweep(args, world, rank, dev, sn):
    """The protocol of the paper's scaling benchmarks (Sec. 4) on one GPU:
    NVT at 300 K (Nose-Hoover), 210 MD steps, wall time of the last 100, on
    4,608 and 12,960 atoms of SiO2 at the alpha-quartz density, r_c 4 A,
    2-5 layers, channels 4-64 per irrep (fewer than 32 run as the exact
    zero-padded 32-channel model), lmax 3 as in the paper and lmax 2.  One
    JSON line per configuration and precision."""
    import numpy as np
    import torch
    from synth import benchmark_model, make_quartz, maxwell_boltzmann, normal_weights
    from synth.configs import MASSES_AMU
    masses = np.asarray(MASSES_AMU)
    for cell_name in ("quartz_4608", "quartz_12960"):
        s = make_quartz(cell_name)
        vel = maxwell_boltzmann(masses[s.species], 300.0, seed=12)
        for lmax, n_layers, channels in [(l, n, c) for l in (3, 2) for n in (2, 3, 4, 5) for c in (4, 8, 16, 32, 64)]:
            if True:
                spec = benchmark_model(n_layers, channels, lmax=lmax)
                model = sn.SevenNet(spec, normal_weights(sn.n_params(spec)), device=dev.index)
                for prec in ("fp32", "bf16"):
                    md = sn.MD(model, s.pos, vel, s.species, masses, s.cell, prec)
                    md.set_nose_hoover(300.0, 100.0)
                    md.step(110, 1.0)
                    barrier(world)
                    torch.cuda.synchronize(dev)
                    t0 = time.perf_counter()
                    md.step(100, 1.0)
                    torch.cuda.synchronize(dev)
                    wall = max_over_ranks(time.perf_counter() - t0, world, dev)
                    md.close()
                    line = {"metric": "atom-steps/s (NVT MD, paper benchmark protocol)",
                            "value": world * s.n_atoms * 100 / wall, "unit": UNIT, "n_gpus": world,
                            "steps": 100, "warmup": 110, "ms_per_step": wall * 10.0,
                            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                            "dtype": "f32" if prec == "fp32" else "bf16+f32", "data": "synthetic",
                            "config": {"workload": cell_name, "n_atoms": s.n_atoms, "n_layers": n_layers,
                                       "channels": channels, "lmax": lmax, "r_cut": 4.0, "precision": prec,
                                       "ensemble": "NVT Nose-Hoover 300 K, tau 100 fs", "dt_fs": 1.0,
                                       "parallelism": f"replicas x{world}"}}
                    if rank == 0:
                        print(json.dumps(line), flush=True)
                model.close()


def run_reference(args, world, rank):
    if rank != 0:
        return
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample(steps=1)
    base, _ = oracle_sample(steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 192.0 / base["value"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "192-atom SiO2 cell, same model"},
            "cpu_baseline": base, "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-compare", action="store_true", help="skip the other precision's line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--no-md", action="store_true", help="skip the MD legs of the default run")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--md-steps", type=int, default=0, help="run MD for this many timed steps instead")
    ap.add_argument("--skin", type=float, default=0.0, help="MD: Verlet-list skin in A (0: rebuild every step)")
    ap.add_argument("--nvt", type=float, default=0.0, help="MD: Nose-Hoover target temperature in K (0: NVE)")
    ap.add_argument("--tau", type=float, default=100.0, help="MD: Nose-Hoover time constant in fs")
    ap.add_argument("--melt-quench", type=float, default=0.0,
                    help="run the melt-quench schedule of Sec. 5.2 with every duration times this factor "
                         "(default workload: the 112,000-atom Si3N4 cell)")
    ap.add_argument("--paper-sweep", action="store_true",
                    help="the paper's benchmark protocol (Sec. 4) over the supported model shapes")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch
    import paper_2402_03789_gb300 as sn
    from synth import make_workload, normal_weights

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.paper_sweep:
        paper_sweep(args, world, rank, dev, sn)
        return
    if args.melt_quench > 0 and args.workload == WORKLOAD:
        args.workload = "si3n4_112000"
    s, spec = make_workload(args.workload)
    weights = normal_weights(sn.n_params(spec))
    model = sn.SevenNet(spec, weights, device=local)
    if args.md_steps > 0:
        md_run(args, world, rank, dev, sn, model, s)
        return
    if args.melt_quench > 0:
        melt_quench_run(args, world, rank, dev, sn, model, s)
        return
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    species = torch.tensor(s.species, dtype=torch.int32, device=dev)
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    off = [0, s.n_atoms]
    cells = s.cell[None]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    n_edges = len(model.neighbors(s.pos, s.cell)[0])

    def timed(prec):
        out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((s.n_atoms, 3), dtype=torch.float64, device=dev),
               torch.empty((1, 3, 3), dtype=torch.float64, device=dev))
        for _ in range(args.warmup):
            model.evaluate_batch_dev(off, cells, species, pos, prec, stream=stream, out=out)
        torch.cuda.synchronize(dev)
        model.profile(True)
        l0 = sn.SevenNet.launch_count()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clk = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clk.start()
        w0 = time.perf_counter()
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            model.evaluate_batch_dev(off, cells, species, pos, prec, stream=stream, out=out)
            b.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        wall = time.perf_counter() - w0
        clk.stop()
        per_step = [a.elapsed_time(b) for a, b in evs]
        dev_ms = sum(per_step)
        prof = model.profile_read()
        model.profile(False)
        launches = sn.SevenNet.launch_count() - l0
        dev_ms = max_over_ranks(dev_ms, world, dev)
        med_ms = max_over_ranks(statistics.median(per_step), world, dev)
        return dev_ms, wall, prof, launches, clk.summary(), out, med_ms

    dev_ms, wall, prof, launches, clocks, out, med_ms = timed(args.precision)
    value = world * s.n_atoms * args.steps / (dev_ms / 1e3)
    ms_per_step = dev_ms / args.steps

    # e2e: the host-buffer C-ABI call, copies included, every step
    e2e_t = []
    model.evaluate(s.pos, s.cell, s.species, args.precision)
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        model.evaluate(s.pos, s.cell, s.species, args.precision)
        e2e_t.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(statistics.median(e2e_t), world, dev)
    h2d = s.n_atoms * 3 * 8 + s.n_atoms * 4 + 9 * 8
    d2h = 8 + s.n_atoms * 3 * 8 + 9 * 8

    # roofline of the dominant kernel family (the convolution adjoint)
    fam = max(("conv_bwd", "conv_fwd"), key=lambda k: prof.get(k, (0, 0))[0])
    tot_ms, n_launch = prof[fam]
    tc = args.precision == "bf16"
    per = [conv_flops_per_edge(spec, t, fam == "conv_bwd", tc) for t in range(spec.n_layers)]
    alu_step = sum(a for a, _ in per) * n_edges
    tc_step = sum(b for _, b in per) * n_edges
    achieved = alu_step * args.steps / (tot_ms / 1e3) / 1e12
    alu = measure_alu_peak(sn, local)
    peak = alu["peak_tflops"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_for(fam) if args.workload == WORKLOAD and tc else None,
                "kernel": fam, "share_of_step": tot_ms / dev_ms,
                "peak_source": "measured FP32 FMA throughput (of measured; sevennet_fp32_peak, best of the "
                               "scalar and packed forms)", "alu_peak": alu,
                "peak_from_unit_counts": fp32_alu_peak_tflops(n_sm, 2070.0),
                "alu_flops_per_step": alu_step}
    if tc:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        t_ach = tc_step * args.steps / (tot_ms / 1e3) / 1e12
        roofline["tensor"] = {"achieved": t_ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                              "frac": t_ach / peaks["bf16_tflops"], "flops_per_step": tc_step,
                              "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "median_ms_per_step": med_ms,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == WORKLOAD else args.workload,
                       "n_atoms": s.n_atoms, "n_edges": n_edges, "precision": args.precision,
                       "model": "5-layer 128x0e+64x1e+32x2e lmax 2, r_c 5 A, MLP 8-64-64 (random FP64 weights)",
                       "l2": "256 MB buffer zeroed between timed steps", "parallelism": f"replicas x{world}"},
            "e2e": {"value": world * s.n_atoms / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "wall_ms_per_step": wall * 1e3 / args.steps}

    if not args.no_compare:
        other = "fp32" if args.precision == "bf16" else "bf16"
        o_ms, *_ = timed(other)
        line["compare"] = {other: {"value": world * s.n_atoms * args.steps / (o_ms / 1e3),
                                   "ms_per_step": o_ms / args.steps}}

    if not args.no_serving and rank == 0:
        line["serving"] = serving_run(sn, model, args.precision)
        # offered load far above capacity: the server's own throughput and latency, both precisions
        line["serving_saturated"] = {p: serving_run(sn, model, p, rate_hz=20000.0) for p in ("bf16", "fp32")}

    if not args.no_md and rank == 0 and args.workload == WORKLOAD:
        # the MD configurations: 100 FP32 NVE steps of 3,000 atoms and 20 BF16 NVE steps of 112,000 atoms
        line["md"] = {"sio2_3000_fp32": md_leg(sn, model, "sio2_3000", "fp32", 100, device=local),
                      "si3n4_112000_bf16": md_leg(sn, model, "si3n4_112000", "bf16", 20, device=local)}

    if rank == 0 and world == 1 and not args.no_cpu:
        base, (s2, spec2, w2, res) = oracle_sample()
        line["cpu_baseline"] = base
        # error of each GPU path on the same 192-atom cell, against the oracle's result
        Eo, Fo, Wo = res[0], res[1], res[2]
        m2 = sn.SevenNet(spec2, w2, device=local)
        errs = {}
        for prec in ("fp32", "bf16"):
            E, F, W = m2.evaluate(s2.pos, s2.cell, s2.species, prec)
            errs[prec] = {"force_rel_rms": float(np.linalg.norm(F - Fo) / np.linalg.norm(Fo)),
                          "energy_per_atom_ev": abs(E - Eo) / s2.n_atoms,
                          "virial_rel": float(np.linalg.norm(W - Wo) / np.linalg.norm(Wo))}
        line["error_vs_oracle_192"] = errs
        m2.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
