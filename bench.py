#!/usr/bin/env python
"""VV10 pair-evaluation throughput on GB300 (and the FP64 CPU oracle as the reference arm).

One step = one pass of the whole hot path over the workload's synthetic grid, through the
C ABI: vv10_prepare_points -> vv10_evaluate (energy, potential, Hessian contraction with P
trials, point gradient, atom sums; atom-resolved E/U/W^Bgr on the grids small enough to keep
them).  Every quantity of the step is a sum over all N_kept^2 ordered pairs, so
    value = N_kept^2 * steps / (time of the timed steps)             [pair evals/s]
with inputs resident in HBM when the timed region starts.  The metric's two quantities are
also timed on their own entry points (metric_parts: energy + potential, Hessian
contraction), each beside its FP64 rate on the same GPU.  Default workload: the 60-atom CHON
molecule (1,359,000 points, P = 180), mixed precision with the split-FP16 contraction.
N > 1 (torchrun): every rank runs its own copy of the workload (independent problems, no
data-path collective); value sums over ranks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload chon60|hexamer|water|cluster24|batch]
                       [--precision f16x3|tf32x3|fp64]
--workload batch runs the 64-molecule batch through vv10_batch_prepare + vv10_batch_run
(energy, potential and Hessian contraction; 2 sum_m N_kept,m^2 pairs per step); the default
run adds the same batch as a second record ("batch": 3 timed steps, split TF32, its own
roofline, FP64 comparison on a subset and end-to-end timing).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "VV10 pair evals/s: E+potential & Hessian contraction, mixed vs FP64 GPU"
UNIT = "pair evals/s"
DTYPES = {"f16x3": "f32 pair tiles, split-fp16 tensor-core contraction, f64 precompute/reductions",
          "mixed": "f32 pair tiles, split-tf32 tensor-core contraction, f64 precompute/reductions",
          "tf32x3": "f32 pair tiles, split-tf32 tensor-core contraction, f64 precompute/reductions",
          "fp64": "f64",
          "fp64tc": "f64 pair sums; Hessian contraction from double-fp32 tiles cut into 8-bit "
                    "integer slices, exact fp32 tensor-core level sums"}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128
# FP32 operations per pair counted from the formulas each kernel evaluates:
#   tensor-core contraction: kernel tiles T1..T4 (36, the reciprocal counted once) and
#   their four hi - lo subtractions
ALU_OPS_PER_PAIR_TC = 40
# the same when each output kind has its own tile generation (Ppad > 64): 2 x (25 + 5.5 + 2)
ALU_OPS_PER_PAIR_TC_SPLIT = 65
#   plain energy/potential pass: 13 shared (R^2, g, g', s, g g' s, reciprocal with its Newton
#   step, Phi c) + 7 (1/s + 1/g and the three sums)
ALU_OPS_PER_PAIR_EUW = 20
#   grid-grid Hessian block D_i^B: the same 13 shared, 10 for 1/(g g'), 1/s, omega_i/g,
#   omega_j/g', (omega_i+omega_j)/s and D, 4 for the squared bracket, 4 for the scaled
#   displacement, 6 outer-product and 1 identity-term accumulations
ALU_OPS_PER_PAIR_CH = 38
#   weight-derivative sums: 19 to form 1/(g g' s), 1/s + 1/g and the three kernel values,
#   then 3 FMAs per direction
ALU_OPS_PER_PAIR_WR = 19
#   FP64 tensor-core contraction, per pair, trial group of 32 and output kind: 33 for the
#   exact coordinate differences and r^2, about 250 for the double-FP32 kernel tiles (17
#   additions of 11 operations, 24 products of 7, a reciprocal of 12), 2 x 30 for the seven
#   slices of the two tiles, and 8 x 40 / 4 for the level drains of the row's outputs
#   (shared by the 4 j a thread generates per stage); both output kinds
O64_ALU_OPS_PER_PAIR = 2 * (33 + 250 + 60 + 80)
# DRAM bytes per launch of the dominant kernel from one ncu capture of the current kernel on
# the full-size launch, keyed by (kernel, workload); absent -> traffic null.
PROFILED_TRAFFIC = {
    # k_hess_f16 on the 60-atom grid (P = 180, one 192-wide group, 24 MB j chunks, evict-last
    # trial tiles, streaming partial output): ncu dram__bytes_read.sum + dram__bytes_write.sum
    # of one launch
    ("k_hess_f16", "chon60"): 630.09e9 + 194.94e9,
}


def workloads():
    from paper_2208_14639_gb300 import synth
    return {
        "water": ("water, 3 atoms, 30x110 points per atom (9,900 points), P=9", synth.config_water),
        "hexamer": ("water-hexamer-like cluster, 18 atoms, 50x194 points per atom (174,600 points), P=54",
                    synth.config_water_hexamer),
        "cluster24": ("24-atom fragment cluster, 30x139 points per atom (100,080 points), P=72",
                      synth.config_cluster24),
        "chon60": ("60-atom CHON molecule, 75x302 points per atom (1,359,000 points), P=180",
                   synth.config_chon60),
        # the same molecule on a coarser grid: P = 180 at a device footprint of a few GB
        "chon60s": ("60-atom CHON molecule, 40x110 points per atom (264,000 points), P=180",
                    lambda: synth.config_chon60(n_rad=40, n_ang=110)),
    }


# Largest grid on which the breakdown also times the weight-derivative sums and the AO-side
# assembly (their host-side inputs grow as N x N_atom and N x nbf).
EXTRA_CALLS_MAX_POINTS = 400_000

# Radial x angular points per atom of each workload's grid (for its weight derivatives).
GRID_SHAPES = {"water": (30, 110), "hexamer": (50, 194), "cluster24": (30, 139),
               "chon60": (75, 302), "chon60s": (40, 110)}


# ------------------------------------------------------------------ host-side rank logic

def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment (defaults 0, 1, 0)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of a per-rank scalar (a host-side reduction of the timing, not of data)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "-i", str(self.index),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, active = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.REASONS, parts[2:6]):
                if v.lower().startswith("active"):
                    active.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(active),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm

def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


class Problem:
    """A workload's inputs resident on the device plus preallocated outputs.  Trial densities
    are evaluated on the device (the same formulas as the host generator); `host` holds the
    step's inputs in host memory (the trials copied back once, untimed) for the end-to-end
    timing and the oracle."""

    def __init__(self, g, dev, resolved: bool = True):
        import torch
        from paper_2208_14639_gb300 import synth
        T = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        self.g = g
        self.n = g.n
        self.n_atom = g.molecule.n_atom
        self.d = {"xyz": T(g.coords), "w": T(g.weights), "rho": T(g.rho), "grad": T(g.grad_rho),
                  "atom": T(g.atom_of_point, torch.int32)}
        self.d["rt"], self.d["gt"] = synth.trial_densities_torch(g.molecule, self.d["xyz"])
        self.P = int(self.d["rt"].shape[0])
        self.host = {"xyz": g.coords, "w": g.weights, "rho": g.rho, "grad": g.grad_rho,
                     "atom": g.atom_of_point.astype(np.int32),
                     "rt": self.d["rt"].cpu().numpy(), "gt": self.d["gt"].cpu().numpy()}
        f64 = dict(dtype=torch.float64, device=dev)
        self.out = {
            "vrho": torch.empty(self.n, **f64), "vgamma": torch.empty(self.n, **f64),
            "frt": torch.empty(self.P, self.n, **f64), "fgt": torch.empty(self.P, self.n, **f64),
            "gp": torch.empty(self.n, 3, **f64), "ga": torch.empty(self.n_atom, 3, **f64),
            # atom-resolved terms (3 x n x n_atom x 3 FP64; 5.9 GB on the 60-atom grid, so
            # that workload leaves them out and takes the point gradient from its own pass)
            "euw": torch.empty(3, self.n, self.n_atom, 3, **f64) if resolved else None,
        }

    def weight_dirs(self):
        """The 3 N_atom nuclear derivatives of the Becke weights (P x n, on the device); made
        on first use (a few seconds of host work), for the grids whose recipe is known."""
        import torch
        if getattr(self, "_wdirs", None) is None:
            from paper_2208_14639_gb300 import synth
            V = synth.weight_directions(self.g.molecule, *self.grid_shape)
            self._wdirs = torch.from_numpy(V).to(self.d["xyz"].device)
        return self._wdirs

    def input_bytes(self):
        return int(sum(v.nbytes for v in self.host.values()))


def run_step(vv, h, pb, prec, d=None, o=None, want_energy=True):
    """One pass of the whole path through the C ABI (prepare, then energy, potential, Hessian
    contraction and coordinate terms in one vv10_evaluate call); returns (n_kept, energy).
    d, o: the device input and output tensors (default: the problem's own)."""
    d = pb.d if d is None else d
    o = pb.out if o is None else o
    nk = vv.vv10_prepare_points(h, d["xyz"], d["w"], d["rho"], d["grad"], d["atom"], pb.n_atom)
    e = vv.vv10_evaluate(h, prec, d["rt"], d["gt"], o["frt"], o["fgt"], vrho=o["vrho"],
                         vgamma=o["vgamma"], grad_points=o["gp"], grad_atoms=o["ga"],
                         EUW_Bgr=o["euw"], want_energy=want_energy)
    return nk, e


def time_steps(vv, h, pb, prec, steps, warmup, world):
    import torch
    for _ in range(warmup):
        run_step(vv, h, pb, prec)
    vv.vv10_sync(h)
    vv.vv10_profile_enable(h, True)
    vv.vv10_profile_read(h)  # reset counters
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    nk = e = None
    for _ in range(steps):
        nk, e = run_step(vv, h, pb, prec)
    b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = a.elapsed_time(b)
    prof = vv.vv10_profile_read(h)
    vv.vv10_profile_enable(h, False)
    return ms, nk, e, prof


def time_calls(vv, h, pb, prec, reps):
    """The two metric quantities on their own, device-resident, after the timed steps: the
    energy + potential call (the plain E/U/W pass and its epilogue) and the Hessian
    contraction call (trial preparation, contraction, epilogue; its A/B/C sums are formed
    by the untimed first call and reused).  Milliseconds per call."""
    import torch
    d, o = pb.d, pb.out
    vv.vv10_set_options(h, 0)
    vv.vv10_prepare_points(h, d["xyz"], d["w"], d["rho"], d["grad"], d["atom"], pb.n_atom)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    vv.vv10_energy_potential(h, prec, o["vrho"], o["vgamma"], want_energy=False)
    vv.vv10_hessian_contract(h, prec, d["rt"], d["gt"], o["frt"], o["fgt"])
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        vv.vv10_energy_potential(h, prec, o["vrho"], o["vgamma"], want_energy=False)
    ev[1].record(stream)
    vv.vv10_hessian_contract(h, prec, d["rt"], d["gt"], o["frt"], o["fgt"])  # A/B/C of this pass
    torch.cuda.synchronize()
    ev[2].record(stream)
    for _ in range(reps):
        vv.vv10_hessian_contract(h, prec, d["rt"], d["gt"], o["frt"], o["fgt"])
    ev[3].record(stream)
    torch.cuda.synchronize()
    vv.vv10_set_options(h, vv.VV10_OPT_FUSE_HESSIAN_SUMS)  # as the step runs
    return ev[0].elapsed_time(ev[1]) / reps, ev[2].elapsed_time(ev[3]) / reps


def coord_hessian_pairs(pb):
    """Pairs the grid-grid Hessian blocks need: the unordered pairs {i, j} of kept points of
    different atoms (the pair term is symmetric, so E^{BA} = E^{AB})."""
    kept = pb.host["rho"] >= 1e-10
    n_a = np.bincount(pb.host["atom"][kept], minlength=pb.n_atom).astype(np.float64)
    return float(n_a.sum() ** 2 - (n_a ** 2).sum()) / 2.0


def time_coord_hessian(vv, h, pb, prec, reps):
    """The grid-grid nuclear Hessian block (vv10_coord_hessian, the E^{AB}_{gr,gr} blocks
    only) on the prepared points, device-resident: milliseconds per call."""
    import torch
    E = torch.empty(pb.n_atom, pb.n_atom, 3, 3, dtype=torch.float64, device=pb.d["xyz"].device)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    vv.vv10_coord_hessian(h, prec, E, None)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        vv.vv10_coord_hessian(h, prec, E, None)
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


def time_energy_only(vv, h, prec, reps):
    """vv10_energy (the energy from the unordered pairs) on the prepared points: ms per call
    (each call ends with the host read of the energy)."""
    import torch
    vv.vv10_energy(h, prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        vv.vv10_energy(h, prec)
    return (time.perf_counter() - t0) * 1e3 / reps


def time_weight_response(vv, h, pb, prec, V, reps):
    """The weight-derivative sums (vv10_weight_response) for the directions V (P x n, on the
    device) on the prepared points: milliseconds per call."""
    import torch
    E, U, W = (torch.empty_like(V) for _ in range(3))
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    vv.vv10_weight_response(h, prec, V, E, U, W)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        vv.vv10_weight_response(h, prec, V, E, U, W)
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


def weight_response_roofline(prec, P, pairs, ms, alu_peak_ops, peaks):
    """Roofline view of one weight-derivative call: 6 P algorithmic flops per pair (three
    kernel matrices times P directions).  The mixed path from 5 directions up runs on tensor
    cores: 3 split products x 2 x 3 x Ppad issued flops per pair against the tf32 dense peak;
    otherwise FP32 ALU work (19 + 3 P operations per pair) against the ALU peak."""
    from paper_2208_14639_gb300 import vv10 as vv
    t = ms / 1e3
    out = {"weight_response_alg_tflops": 6.0 * P * pairs / t / 1e12}
    if prec != vv.VV10_FP64 and P > 4:
        groups = -(-P // 64)
        pg = -(-P // groups)
        ppad = 32 if pg <= 32 else 64
        tf32_peak = peaks["bf16_tflops"] * 0.5 * 1e12
        out["weight_response_issued_mma_frac"] = 3 * 6.0 * ppad * groups * pairs / t / tf32_peak
        out["weight_response_tc_alu_frac"] = 28.0 * groups * pairs / t / alu_peak_ops
    else:
        out["weight_response_alu_frac"] = (ALU_OPS_PER_PAIR_WR + 3 * P) * pairs / t / alu_peak_ops
    return out


def time_ao_assembly(vv, h, pb, reps):
    """The AO-side assembly (vv10_fock_matrix, vv10_orbital_hessian) of the step's outputs with
    the synthetic Gaussian basis of the molecule on the grid: (ms per Fock matrix, ms per
    orbital-Hessian call for the P trials, nbf)."""
    import torch
    from paper_2208_14639_gb300 import synth
    basis = synth.ao_basis(pb.g.molecule)
    phi, dphi = synth.ao_values(basis, pb.host["xyz"])
    dev = pb.d["xyz"].device
    phi, dphi = torch.from_numpy(phi).to(dev), torch.from_numpy(dphi).to(dev)
    o, d = pb.out, pb.d
    nbf = basis.nbf
    F = torch.empty(nbf, nbf, dtype=torch.float64, device=dev)
    G = torch.empty(pb.P, nbf, nbf, dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    stream = torch.cuda.current_stream()
    vv.vv10_fock_matrix(h, phi, dphi, o["vrho"], o["vgamma"], F)
    vv.vv10_orbital_hessian(h, phi, dphi, o["frt"], o["fgt"], d["gt"], o["vgamma"], G)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        vv.vv10_fock_matrix(h, phi, dphi, o["vrho"], o["vgamma"], F)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(reps):
        vv.vv10_orbital_hessian(h, phi, dphi, o["frt"], o["fgt"], d["gt"], o["vgamma"], G)
    ev[3].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps, ev[2].elapsed_time(ev[3]) / reps, nbf


def time_fock_derivative(vv, h, pb, prec, wdirs, reps):
    """The nuclear derivative of the Fock matrix (vv10_fock_derivative) along the step's 3 N_atom
    trial directions, with the weight-derivative sums along the Becke weight directions, the
    step's atom-resolved sums and the synthetic Gaussian basis (values, gradients, Hessians) on
    the grid: milliseconds per call (each call reads the atom segments back to the host)."""
    import torch
    from paper_2208_14639_gb300 import synth
    o, d = pb.out, pb.d
    if o["euw"] is None:
        return None
    basis = synth.ao_basis(pb.g.molecule)
    xyz = pb.host["xyz"]
    dev = d["xyz"].device
    phi, dphi = (torch.from_numpy(x).to(dev) for x in synth.ao_values(basis, xyz))
    d2phi = torch.from_numpy(synth.ao_second_derivatives(basis, xyz)).to(dev)
    bf_atom = torch.from_numpy(basis.atom.astype(np.int32)).to(dev)
    E, U, W = (torch.empty_like(wdirs) for _ in range(3))
    vv.vv10_weight_response(h, prec, wdirs, E, U, W)
    nbf = basis.nbf
    FA = torch.empty(3 * pb.n_atom, nbf, nbf, dtype=torch.float64, device=dev)
    args = (h, phi, dphi, d2phi, bf_atom, o["vrho"], o["vgamma"], o["frt"], o["fgt"], d["gt"],
            wdirs, E, U, W, o["euw"], FA)
    vv.vv10_fock_derivative(*args)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        vv.vv10_fock_derivative(*args)
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


def time_e2e(vv, h, pb, prec, steps, warmup):
    """The same step with host inputs: every step copies all of its inputs from pinned host
    memory to the device and all of its outputs back, inside the timed region.  The copies
    run on a second stream, pipelined with the computation over two device buffer sets: the
    inputs of step k+1 arrive and the outputs of step k leave while the next step computes."""
    import torch
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).to(
        torch.int32 if k == "atom" else torch.float64).pin_memory() for k, v in pb.host.items()}
    pout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in pb.out.items()
            if v is not None}
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    d2h = sum(t.numel() * t.element_size() for t in pout.values())
    sets = [pb.d, {k: torch.empty_like(v) for k, v in pb.d.items()}]
    outs = [pb.out, {k: (None if v is None else torch.empty_like(v)) for k, v in pb.out.items()}]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()

    def run(n):
        ev_in, ev_done, ev_out = {}, {}, {}
        nk = 0

        def h2d_into(k):
            with torch.cuda.stream(copy):
                if k >= 2:
                    copy.wait_event(ev_done[k - 2])  # the set's last reader
                for key, t in pin.items():
                    sets[k % 2][key].copy_(t, non_blocking=True)
                ev_in[k] = torch.cuda.Event()
                ev_in[k].record(copy)

        h2d_into(0)
        for k in range(n):
            if k + 1 < n:
                h2d_into(k + 1)
            comp.wait_event(ev_in[k])
            if k >= 2:
                comp.wait_event(ev_out[k - 2])  # the set's outputs have left
            nk, _ = run_step(vv, h, pb, prec, sets[k % 2], outs[k % 2], want_energy=False)
            ev_done[k] = torch.cuda.Event()
            ev_done[k].record(comp)
            with torch.cuda.stream(copy):
                copy.wait_event(ev_done[k])
                for key, t in pout.items():
                    t.copy_(outs[k % 2][key], non_blocking=True)
                ev_out[k] = torch.cuda.Event()
                ev_out[k].record(copy)
        return nk

    run(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nk = run(steps)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return sec, nk, h2d, d2h


def oracle_rows(args, rt, gt, rows):
    """The oracle's whole path for a set of rows i (full j sums): potential, Hessian
    contraction with every trial, point gradient."""
    import oracle
    oracle.potential(*args, rows=rows)
    oracle.hessian_contract(*args, rt, gt, rows=rows)
    oracle.point_grad(*args, rows=rows)


def cpu_baseline(pb, budget_s: float):
    """The FP64 oracle, as it stands, on a bounded row sample of the same workload: each
    sampled row runs the whole path over all j, so a row counts N_kept pairs."""
    import oracle
    g = pb.g
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = np.flatnonzero(g.rho >= 1e-10)
    nk = kept.size
    cores = len(os.sched_getaffinity(0))
    oracle.set_num_threads(cores)
    # calibrate on a small sample, then size the sample to the budget
    rows = kept[np.linspace(0, nk - 1, 16).astype(np.int64)]
    t0 = time.perf_counter()
    oracle_rows(args, pb.host["rt"], pb.host["gt"], rows)
    cal = time.perf_counter() - t0
    n_rows = int(min(nk, max(16, 16 * budget_s / max(cal, 1e-3))))
    rows = kept[np.linspace(0, nk - 1, n_rows).astype(np.int64)]
    t0 = time.perf_counter()
    oracle_rows(args, pb.host["rt"], pb.host["gt"], rows)
    sec = time.perf_counter() - t0
    return {"value": n_rows * nk / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": sec,
            "sample": f"{n_rows} rows of {nk} kept points, each through the whole path "
                      f"(potential, Hessian contraction with P={pb.P}, point gradient), full j sums"}


def fp64_hessian_same_grid(vv, dev, prec):
    """FP64 (SIMT and tensor-core integer slices) against mixed Hessian contraction on the
    water-hexamer grid (174,600 points, P = 54): on the larger grids the FP64 SIMT contraction
    alone would take many minutes.  Each call timed once after an untimed one; milliseconds,
    pairs per second and the distance of each result to the FP64 SIMT one."""
    import torch
    from paper_2208_14639_gb300 import synth
    g = synth.config_water_hexamer()
    pb = Problem(g, dev, resolved=False)
    h = vv.vv10_create(dev.index or 0)
    d, o = pb.d, pb.out
    nk = vv.vv10_prepare_points(h, d["xyz"], d["w"], d["rho"], d["grad"], d["atom"], pb.n_atom)
    out = {"workload": "water-hexamer-like cluster, 174,600 points, P=54", "n_kept": nk}
    stream = torch.cuda.current_stream()
    res = {}
    for name, p in (("mixed", prec), ("fp64", vv.VV10_FP64), ("fp64tc", vv.VV10_FP64_TC)):
        vv.vv10_energy_potential(h, p, o["vrho"], o["vgamma"], want_energy=False)
        vv.vv10_hessian_contract(h, p, d["rt"], d["gt"], o["frt"], o["fgt"])
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        vv.vv10_hessian_contract(h, p, d["rt"], d["gt"], o["frt"], o["fgt"])
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        out[f"{name}_ms"] = ms
        out[f"{name}_pair_evals_per_s"] = float(nk) * nk / (ms / 1e3)
        res[name] = (o["frt"].clone(), o["fgt"].clone())
    out["speedup_mixed_vs_fp64"] = out["fp64_ms"] / out["mixed_ms"]
    out["speedup_fp64tc_vs_fp64"] = out["fp64_ms"] / out["fp64tc_ms"]
    for name in ("mixed", "fp64tc"):  # relative Frobenius distance to the FP64 SIMT result
        out[f"{name}_rel_diff_vs_fp64"] = max(
            float(torch.linalg.norm(res[name][k] - res["fp64"][k]) / torch.linalg.norm(res["fp64"][k]))
            for k in range(2))
    vv.vv10_destroy(h)
    return out


def gpu_arm(args):
    import torch
    from paper_2208_14639_gb300 import vv10 as vv

    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vv.load(build_if_missing=True)
    label, make = workloads()[args.workload]
    g = make()
    pb = Problem(g, dev, resolved=not args.workload.startswith("chon60"))
    pb.grid_shape = GRID_SHAPES[args.workload]
    h = vv.vv10_create(local)
    prec = vv.PRECISIONS[args.precision]
    peaks, peak_src = load_peaks()
    large = pb.n > EXTRA_CALLS_MAX_POINTS
    # the step runs the Hessian after the energy: form A/B/C in the energy pass
    vv.vv10_set_options(h, vv.VV10_OPT_FUSE_HESSIAN_SUMS)
    if prec not in (vv.VV10_FP64, vv.VV10_FP64_TC):  # tile shapes tuned on first use (warm-up)
        vv.vv10_set_autotune(h, vv.VV10_TUNE_PAIRSUMS | vv.VV10_TUNE_CONTRACTION)

    with ClockSampler(local) as clk:
        ms, nk, e_mixed, prof = time_steps(vv, h, pb, prec, args.steps, args.warmup, world)
    tiles = {"pair_sums_rows_per_thread_splits": [vv.vv10_get_tiles(h, m) for m in range(3)],
             "fused_energy_abc_pass": True,
             "contraction_group_width": vv.vv10_get_tiles(h, vv.TILES_CONTRACTION)[0]}
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world)
    pairs_call = float(nk) * float(nk)
    # every quantity of the step is a sum over all N_kept^2 ordered pairs: value counts each
    # pair once per step
    value = pairs_call * args.steps * world / (ms_max / 1e3)

    K = args.steps
    per = {k: v[0] / K for k, v in prof.items()}
    launches = sum(v[1] for v in prof.values())
    t_coord = per["pair_sums_grad"] + per["grad_epilogue"] + per["atom_resolved"]  # incl. the fused sums
    hess_flops = 8.0 * pairs_call * pb.P
    ms_ep, ms_hc = time_calls(vv, h, pb, prec, 3)
    ms_e = time_energy_only(vv, h, prec, 3)
    alu_peak_ops = N_SM * FP32_LANES_PER_SM * (clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    breakdown = {
        # the energy alone from the unordered pairs (vv10_energy; half the pair evaluations)
        "energy_only_call_ms": ms_e,
        "energy_only_pairs_per_s": pairs_call / (ms_e / 1e3),
    }
    if not large:  # the calls beyond the step, on grids whose host-side inputs stay small
        ms_ch = time_coord_hessian(vv, h, pb, prec, 3)
        pairs_ch = coord_hessian_pairs(pb)
        wdirs = pb.weight_dirs()
        P_w = int(wdirs.shape[0])
        ms_wr = time_weight_response(vv, h, pb, prec, wdirs, 3)
        ms_fock, ms_gt, nbf = time_ao_assembly(vv, h, pb, 3)
        ms_fa = time_fock_derivative(vv, h, pb, prec, wdirs, 3)
        breakdown.update({
            # the grid-grid nuclear Hessian block (not part of the step)
            "coord_hessian_call_ms": ms_ch,
            "coord_hessian_pairs": pairs_ch,
            "coord_hessian_pairs_per_s": pairs_ch / (ms_ch / 1e3),
            "coord_hessian_alu_frac": ALU_OPS_PER_PAIR_CH * pairs_ch / (ms_ch / 1e3) / alu_peak_ops,
            # AO-side assembly of the step's outputs (not part of the step): 2 nbf^2 flops per
            # point and channel
            "ao_nbf": nbf,
            "fock_matrix_call_ms": ms_fock,
            "orbital_hessian_call_ms": ms_gt,
            "orbital_hessian_fp64_tflops": 2.0 * nbf * nbf * nk * pb.P / (ms_gt / 1e3) / 1e12,
            # nuclear derivative of the Fock matrix (3 N_atom directions): 2 nbf^2 flops per
            # point and direction, plus 24 nbf^2 per point for the basis-function derivatives
            "fock_derivative_call_ms": ms_fa,
            "fock_derivative_fp64_tflops": (2.0 * nbf * nbf * nk * (3 * pb.n_atom + 12) / (ms_fa / 1e3) / 1e12
                                            if ms_fa else None),
            # weight-derivative sums for the 3 N_atom Becke weight directions (not in the step)
            "weight_response_P": P_w,
            "weight_response_call_ms": ms_wr,
            "weight_response_pairs_per_s": pairs_call / (ms_wr / 1e3),
            **weight_response_roofline(prec, P_w, pairs_call, ms_wr, alu_peak_ops, peaks),
        })
    else:
        breakdown["calls_beyond_the_step"] = f"not timed above {EXTRA_CALLS_MAX_POINTS} points"
    breakdown.update({
        "step_pair_pass_pairs_per_s": pairs_call / (t_coord / 1e3) if t_coord else None,
        "phase_ms_per_step": {k: round(v, 4) for k, v in per.items() if v},
        "note": "in the step one pass over the pairs forms the E/U/W and A/B/C row sums and the "
                "point gradient (and, on the grids that keep them, the atom-resolved terms); "
                "then the contraction",
    })

    # the metric's two quantities on their own (each its own entry point, 3 calls each)
    parts = {
        "energy_potential": {
            "pair_evals_per_s": pairs_call / (ms_ep / 1e3), "ms_per_call": ms_ep,
            "alu_frac": ALU_OPS_PER_PAIR_EUW * pairs_call / (ms_ep / 1e3) / alu_peak_ops},
        "hessian_contraction": {
            "pair_evals_per_s": pairs_call / (ms_hc / 1e3), "ms_per_call": ms_hc,
            "P": pb.P, "P_pair_evals_per_s": pb.P * pairs_call / (ms_hc / 1e3),
            "alg_tflops": hess_flops / (ms_hc / 1e3) / 1e12},
        "counting": "ordered pairs sum N_kept^2 per call, independent of the kernels' "
                    "symmetry shortcuts",
    }

    # roofline of the dominant kernel
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    dom = max(per, key=per.get)
    roof = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "kernel": dom}
    if dom == "contraction_tensor_core" and prec == vv.VV10_FP64_TC:
        # FP32 ALU-bound: double-FP32 tile generation, slicing and level drains
        t = per[dom] / 1e3
        groups = -(-pb.P // 32)
        alu_peak = N_SM * FP32_LANES_PER_SM * sm_mhz * 1e6
        ops = O64_ALU_OPS_PER_PAIR * groups * pairs_call
        roof = {"bound": "alu", "achieved": ops / t / 1e12, "peak": alu_peak / 1e12,
                "unit": "Tops/s (FP32)", "frac": ops / t / alu_peak, "traffic": None,
                "kernel": "k_hess_o64",
                "peak_source": f"{N_SM} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz",
                "counting": f"{O64_ALU_OPS_PER_PAIR} FP32 operations per pair and trial group of 32 "
                            "(both output kinds)"}
    elif dom == "contraction_tensor_core":
        t = per[dom] / 1e3
        groups = -(-pb.P // 192)
        ppad = max(32, 32 * -(-(-(-pb.P // groups)) // 32))
        f16 = prec == vv.VV10_MIXED_F16X3
        kernel = "k_hess_f16" if f16 else "k_hess_tc"
        # the dense peak of the operand type: FP16 = the measured bf16 rate (same MMA rate);
        # TF32 = half of it (the nominal ratio).  The contraction runs for seconds inside a
        # long step: the sustained figure.
        key = "bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks else "bf16_tflops"
        peak = peaks[key] * (1.0 if f16 else 0.5) * 1e12
        t_tensor = 3 * 8.0 * pairs_call * ppad * groups / peak
        ops_pair = tc_alu_ops_per_pair(ppad) * groups
        alu_peak = N_SM * FP32_LANES_PER_SM * sm_mhz * 1e6
        roof = {"bound": "tensor", "achieved": hess_flops / t / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": hess_flops / t / peak,
                "traffic": PROFILED_TRAFFIC.get((kernel, args.workload)),
                "kernel": kernel,
                "peak_source": f"{peak_src} {key} {peaks[key]} x {1.0 if f16 else 0.5} "
                               f"({'fp16' if f16 else 'tf32'} dense)",
                "counting": "achieved = 8 P N_kept^2 algorithmic flops per launch / CUDA-event "
                            "time; the 3-product split issues 3 x 8 Ppad N_kept^2",
                "issued_mma_frac": t_tensor / t,
                "alu_alt": {"frac": ops_pair * pairs_call / t / alu_peak, "ops_per_pair": ops_pair}}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES.get(args.precision, "f64"),
        "data": "synthetic (seeded molecule-shaped grids, Gaussian densities, analytic trials)",
        "config": {"workload": label, "n_points": pb.n, "n_kept": nk, "P": pb.P,
                   "precision": args.precision, "pairs_per_step": pairs_call,
                   "value_counts": "N_kept^2 ordered pairs per step: one pass of the whole path "
                                   "(energy, potential, Hessian contraction with P trials, "
                                   "point gradient) over every pair",
                   "l2": f"inputs larger than L2 ({pb.input_bytes() / 1e6:.0f} MB resident)",
                   "parallelism": f"replica x{world}"},
        "metric_parts": parts,
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clocks,
        "breakdown": breakdown,
        "tiles": tiles,
        "energy": e_mixed,
    }

    if rank == 0 and not args.no_fp64_arm and prec not in (vv.VV10_FP64, vv.VV10_FP64_TC):
        vv.vv10_set_autotune(h, 0)  # FP64 baseline at its default shapes
        if not large:
            ms64, nk64, e64, prof64 = time_steps(vv, h, pb, vv.VV10_FP64, 1, 1, 1)
            per64 = {k: v[0] for k, v in prof64.items()}
            ms_ep64, ms_hc64 = time_calls(vv, h, pb, vv.VV10_FP64, 1)
            result["fp64"] = {
                "value": pairs_call / (ms64 / 1e3), "ms_per_step": ms64, "steps": 1, "warmup": 1,
                "energy": e64, "abs_energy_diff_mixed_vs_fp64": abs(e_mixed - e64),
                "phase_ms": {k: round(v, 3) for k, v in per64.items() if v},
            }
            result["speedup_mixed_vs_fp64"] = value / world / result["fp64"]["value"]
            parts["hessian_contraction"]["fp64_pair_evals_per_s"] = pairs_call / (ms_hc64 / 1e3)
            parts["hessian_contraction"]["speedup_vs_fp64"] = ms_hc64 / ms_hc
        else:
            # the FP64 energy/potential call on this grid (one call); the FP64 contraction on
            # the water-hexamer grid, mixed beside it
            o = pb.out
            vv.vv10_prepare_points(h, pb.d["xyz"], pb.d["w"], pb.d["rho"], pb.d["grad"], pb.d["atom"],
                                   pb.n_atom)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e64 = vv.vv10_energy_potential(h, vv.VV10_FP64, o["vrho"], o["vgamma"], want_energy=True)
            ms_ep64 = (time.perf_counter() - t0) * 1e3
            result["fp64"] = {"energy": e64, "abs_energy_diff_mixed_vs_fp64": abs(e_mixed - e64),
                              "energy_potential_ms": ms_ep64,
                              "hessian_contraction_same_grid": fp64_hessian_same_grid(vv, dev, prec)}
        parts["energy_potential"]["fp64_pair_evals_per_s"] = pairs_call / (ms_ep64 / 1e3)
        parts["energy_potential"]["speedup_vs_fp64"] = ms_ep64 / ms_ep

    e2e_steps = K if not large else max(1, min(K, 3))
    sec, nk_e, h2d, d2h = time_e2e(vv, h, pb, prec, e2e_steps, 1)
    result["e2e"] = {"value": pairs_call * e2e_steps / sec, "unit": UNIT, "steps": e2e_steps,
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(pb, args.cpu_seconds)

    vv.vv10_destroy(h)
    if args.with_batch:
        # the 64-molecule batch (many molecules of uneven size in persistent launches and a
        # recorded graph) as a second timed record of the same run, on a freed device
        del pb
        torch.cuda.empty_cache()
        result["batch"] = batch_record(args, dev, world, rank, max(1, min(K, 3)), 2,
                                       args.batch_precision, with_fp64=not args.no_fp64_arm,
                                       with_cpu=False)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ batched workload

BATCH_LABEL = ("64 CHON molecules, 3-30 atoms (uniform), 50x194 points per atom (9,700-291,000 "
               "points each), P = 3 N_atom per molecule")


def tc_alu_ops_per_pair(ppad: int) -> int:
    """FP32 operations per pair of the tensor-core contraction: both outputs share one tile
    generation when Ppad <= 64; above that each output kind generates its own two tiles and
    repeats the common part (25 shared + 7 or 4 tile + 2 split operations per kind)."""
    return ALU_OPS_PER_PAIR_TC if ppad <= 64 else ALU_OPS_PER_PAIR_TC_SPLIT


class BatchProblem:
    """The batch of molecules on the device: concatenated grids, trial densities generated
    on the device (torch), preallocated outputs."""

    def __init__(self, dev, workers: int, systems=None):
        import torch
        from paper_2208_14639_gb300 import synth
        self.sys = systems if systems is not None else synth.config_batch(workers=workers)
        self.P = [3 * g.molecule.n_atom for g in self.sys]
        self.n = [g.n for g in self.sys]
        self.off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.toff = np.concatenate([[0], np.cumsum([P * k for P, k in zip(self.P, self.n)])]).astype(np.int64)
        cat = lambda f: np.ascontiguousarray(np.concatenate([getattr(g, f) for g in self.sys]))
        self.host = {"xyz": cat("coords"), "w": cat("weights"), "rho": cat("rho"),
                     "grad": cat("grad_rho"), "atom": cat("atom_of_point").astype(np.int32)}
        T = lambda a: torch.from_numpy(a).to(dev)
        self.d = {k: T(v) for k, v in self.host.items()}
        tot = int(self.toff[-1])
        f64 = dict(dtype=torch.float64, device=dev)
        self.d["rt"] = torch.empty(tot, **f64)
        self.d["gt"] = torch.empty(tot, 3, **f64)
        for m, g in enumerate(self.sys):
            s, e = int(self.toff[m]), int(self.toff[m + 1])
            synth.trial_densities_torch(g.molecule, self.d["xyz"][int(self.off[m]):int(self.off[m + 1])],
                                        out_rho=self.d["rt"][s:e].view(self.P[m], self.n[m]),
                                        out_grad=self.d["gt"][s:e].view(self.P[m], self.n[m], 3))
        N = int(self.off[-1])
        self.out = {"E": torch.empty(len(self.sys), **f64), "vrho": torch.empty(N, **f64),
                    "vgamma": torch.empty(N, **f64), "frt": torch.empty(tot, **f64),
                    "fgt": torch.empty(tot, **f64)}
        self.n_atom = [g.molecule.n_atom for g in self.sys]

    def input_bytes(self):
        return int(sum(t.numel() * t.element_size() for t in self.d.values()))


def run_batch_step(vv, h, bp, prec):
    """One pass over the whole batch through the C ABI: prepare every molecule, then energy,
    potential and Hessian contraction of all of them (one recorded graph after the first)."""
    d, o = bp.d, bp.out
    nk = vv.vv10_batch_prepare(h, bp.off, d["xyz"], d["w"], d["rho"], d["grad"], d["atom"], bp.n_atom)
    vv.vv10_batch_run(h, prec, bp.P, d["rt"], d["gt"], o["E"], o["vrho"], o["vgamma"], o["frt"], o["fgt"])
    return nk


def time_batch(vv, h, bp, prec, steps, warmup, world):
    import torch
    for _ in range(warmup):
        run_batch_step(vv, h, bp, prec)
    vv.vv10_sync(h)
    vv.vv10_profile_enable(h, True)
    vv.vv10_profile_read(h)
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    nk = None
    for _ in range(steps):
        nk = run_batch_step(vv, h, bp, prec)
    b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    prof = vv.vv10_profile_read(h)
    vv.vv10_profile_enable(h, False)
    return a.elapsed_time(b), nk, prof


def time_batch_e2e(vv, h, bp, prec, steps, warmup):
    """The batched step with host inputs: pinned H2D of every input (grids and trial
    densities) and D2H of every output inside the timed region."""
    import torch
    pin = {k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in bp.d.items()}
    for k, t in pin.items():
        t.copy_(bp.d[k])
    pout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in bp.out.items()}
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    d2h = sum(t.numel() * t.element_size() for t in pout.values())

    def one():
        for k, t in pin.items():
            bp.d[k].copy_(t, non_blocking=True)
        nk = run_batch_step(vv, h, bp, prec)
        for k, t in pout.items():
            t.copy_(bp.out[k], non_blocking=True)
        return nk

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, h2d, d2h


def batch_cpu_sample(bp, budget_s: float):
    """The FP64 oracle on a bounded row sample of the batch: rows of the smallest, a middle
    and the largest molecule (energy/potential and Hessian contraction, full j sums)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_num_threads(cores)
    order = np.argsort(bp.n, kind="stable")
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    data = []
    for m in picks:
        g = bp.sys[m]
        s, e = int(bp.toff[m]), int(bp.toff[m + 1])
        rt = bp.d["rt"][s:e].view(bp.P[m], bp.n[m]).cpu().numpy()
        gt = bp.d["gt"][s:e].view(bp.P[m], bp.n[m], 3).cpu().numpy()
        kept = np.flatnonzero(g.rho >= 1e-10)
        data.append(((g.coords, g.weights, g.rho, g.grad_rho), rt, gt, kept))

    def run(n_rows):
        pairs = 0
        for args, rt, gt, kept in data:
            rows = kept[np.linspace(0, kept.size - 1, n_rows).astype(np.int64)]
            oracle.potential(*args, rows=rows)
            oracle.hessian_contract(*args, rt, gt, rows=rows)
            pairs += 2 * n_rows * kept.size
        return pairs

    t0 = time.perf_counter()
    run(4)
    cal = time.perf_counter() - t0
    n_rows = int(max(4, min(4096, 4 * budget_s / max(cal, 1e-3))))
    t0 = time.perf_counter()
    pairs = run(n_rows)
    sec = time.perf_counter() - t0
    return {"value": pairs / sec, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": sec,
            "sample": f"{n_rows} rows each (energy/potential and Hessian contraction, full j sums) "
                      f"of molecules {picks} ({[bp.n[m] for m in picks]} points, "
                      f"P={[bp.P[m] for m in picks]})"}


def batch_record(args, dev, world, rank, steps, warmup, prec_name, with_fp64=True, with_cpu=True,
                 label_note=None):
    """The 64-molecule batch through vv10_batch_prepare + vv10_batch_run: the timed steps,
    its roofline, the FP64 comparison on a subset, the end-to-end timing and (optionally) the
    oracle sample.  Returns the record (a dict)."""
    import torch
    from paper_2208_14639_gb300 import vv10 as vv
    local = dev.index or 0
    bp = BatchProblem(dev, workers=max(1, len(os.sched_getaffinity(0))))
    h = vv.vv10_create(local)
    prec = vv.PRECISIONS[prec_name]
    peaks, peak_src = load_peaks()
    if prec != vv.VV10_FP64:  # batched pair-sum tiles tuned on first use (warm-up)
        vv.vv10_set_autotune(h, vv.VV10_TUNE_BATCH)

    with ClockSampler(local) as clk:
        ms, nk, prof = time_batch(vv, h, bp, prec, steps, warmup, world)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world)
    nk = np.asarray(nk, dtype=np.float64)
    pairs_step = float((nk * nk).sum())
    K = steps
    value = 2.0 * pairs_step * K * world / (ms_max / 1e3)
    per = {k: v[0] / K for k, v in prof.items()}
    launches = sum(v[1] for v in prof.values())

    # tensor-core groups (<= 192 trials each) and padded group width per molecule
    groups = [-(-p // 192) for p in bp.P]
    ppad = np.array([max(32, 32 * -(-(-(-p // g)) // 32)) for p, g in zip(bp.P, groups)])
    nk2 = nk * nk
    hess_flops = 8.0 * float((nk2 * np.array(bp.P)).sum())
    dom = max(per, key=per.get)
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    roof = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "kernel": dom}
    if dom == "contraction_tensor_core":
        t = per[dom] / 1e3
        f16 = prec == vv.VV10_MIXED_F16X3
        key = "bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks else "bf16_tflops"
        peak = peaks[key] * (1.0 if f16 else 0.5) * 1e12
        t_tensor = 3 * 8.0 * float((nk2 * ppad * np.array(groups)).sum()) / peak
        roof = {"bound": "tensor", "achieved": hess_flops / t / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": hess_flops / t / peak, "traffic": None,
                "kernel": "k_hess_f16 (batched)" if f16 else "k_hess_tc (batched)",
                "peak_source": f"{peak_src} {key} {peaks[key]} x {1.0 if f16 else 0.5}",
                "issued_mma_frac": t_tensor / t}
    t_ep = per["pair_sums_EUW"] + per["energy_epilogue"]
    t_hess = (per["pair_sums_ABC"] + per["trial_prep"] + per["contraction_tensor_core"] +
              per["contraction_fp64"] + per["hessian_epilogue"])
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES.get(prec_name, "f64"),
        "data": "synthetic (seeded CHON molecules, Gaussian densities, analytic trials)",
        "config": {"workload": BATCH_LABEL, "n_molecules": len(bp.sys), "n_points": int(bp.off[-1]),
                   "n_kept": int(nk.sum()), "pairs_per_step": 2.0 * pairs_step,
                   "trials_total": int(sum(bp.P)), "precision": prec_name,
                   "l2": f"inputs larger than L2 ({bp.input_bytes() / 1e9:.1f} GB resident)",
                   "parallelism": f"replica x{world}",
                   "pair_count": "2 sum_m N_kept,m^2 (energy/potential + Hessian contraction)"},
        "roofline": roof, "gpu_launches": launches, "clocks": clocks,
        "tiles": {"batch_rows_per_thread_tiles_per_split": vv.vv10_get_tiles(h, vv.TILES_BATCH)},
        "breakdown": {"energy_abc_pass_pairs_per_s": pairs_step / (t_ep / 1e3) if t_ep else None,
                      "hessian_pairs_per_s": pairs_step / (t_hess / 1e3) if t_hess else None,
                      "hessian_alg_tflops": hess_flops / (t_hess / 1e3) / 1e12 if t_hess else None,
                      "phase_ms_per_step": {k: round(v, 3) for k, v in per.items() if v}},
        "energies_first4": [float(x) for x in bp.out["E"][:4].cpu()],
    }
    if label_note:
        result["note"] = label_note
    if rank == 0 and with_fp64 and prec != vv.VV10_FP64:
        # FP64 baseline on the eight smallest molecules (the whole batch would take minutes)
        vv.vv10_set_autotune(h, 0)
        order = np.argsort(bp.n, kind="stable")[:8]
        sub = BatchProblem(dev, 1, systems=[bp.sys[m] for m in sorted(order)])
        for k in ("rt", "gt"):  # same trial values as the mixed run
            parts = [bp.d[k][int(bp.toff[m]):int(bp.toff[m + 1])] for m in sorted(order)]
            sub.d[k].copy_(torch.cat(parts))
        ms64, nk64, _ = time_batch(vv, h, sub, vv.VV10_FP64, 1, 1, 1)
        e64 = sub.out["E"].cpu().numpy()
        msm, _, _ = time_batch(vv, h, sub, prec, 1, 1, 1)
        em = sub.out["E"].cpu().numpy()
        nk64 = np.asarray(nk64, dtype=np.float64)
        result["fp64_subset"] = {
            "molecules": [int(m) for m in sorted(order)],
            "value": 2.0 * float((nk64 * nk64).sum()) / (ms64 / 1e3),
            "mixed_value_same_subset": 2.0 * float((nk64 * nk64).sum()) / (msm / 1e3),
            "max_abs_energy_diff_mixed_vs_fp64": float(np.abs(em - e64).max()),
        }
        del sub
        run_batch_step(vv, h, bp, prec)  # back to the full batch (the handle holds one batch)
    e2e_steps = max(1, min(K, 2))
    sec, h2d, d2h = time_batch_e2e(vv, h, bp, prec, e2e_steps, 1)
    result["e2e"] = {"value": 2.0 * pairs_step * e2e_steps / sec, "unit": UNIT, "steps": e2e_steps,
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    if rank == 0 and world == 1 and with_cpu:
        result["cpu_baseline"] = batch_cpu_sample(bp, args.cpu_seconds)
    vv.vv10_destroy(h)
    del bp
    return result


def gpu_batch_arm(args):
    import torch
    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2208_14639_gb300 import vv10 as vv
    vv.load(build_if_missing=True)
    result = batch_record(args, dev, world, rank, args.steps, args.warmup, args.batch_precision,
                          with_fp64=not args.no_fp64_arm, with_cpu=not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm (oracle)

def reference_batch_arm(args):
    """The oracle on the batch workload: each step a bounded row sample of three molecules."""
    import oracle
    from paper_2208_14639_gb300 import synth
    systems = synth.config_batch(workers=max(1, len(os.sched_getaffinity(0))))
    n = [g.n for g in systems]
    order = np.argsort(n, kind="stable")
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    cores = len(os.sched_getaffinity(0))
    oracle.set_num_threads(cores)
    data = []
    for m in picks:
        g = systems[m]
        rt, gt = synth.trial_densities(g.molecule, g.coords)
        data.append(((g.coords, g.weights, g.rho, g.grad_rho), rt, gt,
                     np.flatnonzero(g.rho >= 1e-10)))

    def step(n_rows):
        pairs = 0
        for a, rt, gt, kept in data:
            rows = kept[np.linspace(0, kept.size - 1, n_rows).astype(np.int64)]
            oracle.potential(*a, rows=rows)
            oracle.hessian_contract(*a, rt, gt, rows=rows)
            pairs += 2 * n_rows * kept.size
        return pairs

    t0 = time.perf_counter()
    step(4)
    per_step = min(20.0, 120.0 / (args.steps + args.warmup))
    n_rows = int(max(4, min(4096, 4 * per_step / max(time.perf_counter() - t0, 1e-3))))
    for _ in range(args.warmup):
        step(n_rows)
    t0 = time.perf_counter()
    pairs = sum(step(n_rows) for _ in range(args.steps))
    sec = time.perf_counter() - t0
    value = pairs / sec
    sample = (f"{n_rows} rows each (energy/potential and Hessian contraction, full j sums) of "
              f"molecules {picks} ({[n[m] for m in picks]} points) per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": BATCH_LABEL, "n_molecules": len(systems)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def reference_arm(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    if args.workload == "batch":
        return reference_batch_arm(args)
    import oracle
    label, make = workloads()[args.workload]
    g = make()
    from paper_2208_14639_gb300 import synth
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    argsg = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = np.flatnonzero(g.rho >= 1e-10)
    nk = kept.size
    cores = len(os.sched_getaffinity(0))
    oracle.set_num_threads(cores)
    # each step: a bounded row sample, every row through the whole path (about 20 s per step)
    rows = kept[np.linspace(0, nk - 1, 16).astype(np.int64)]
    t0 = time.perf_counter()
    oracle_rows(argsg, rt, gt, rows)
    per_step = min(20.0, 120.0 / (args.steps + args.warmup))
    n_rows = int(min(nk, max(16, 16 * per_step / max(time.perf_counter() - t0, 1e-3))))
    rows = kept[np.linspace(0, nk - 1, n_rows).astype(np.int64)]
    for _ in range(args.warmup):
        oracle_rows(argsg, rt, gt, rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rows(argsg, rt, gt, rows)
    sec = time.perf_counter() - t0
    value = n_rows * nk * args.steps / sec
    sample = (f"{n_rows} rows of {nk} kept points per step, each through the whole path "
              f"(potential, Hessian contraction with P={rt.shape[0]}, point gradient), full j sums")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": label, "n_points": g.n, "n_kept": int(nk),
                                        "P": int(rt.shape[0])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("hexamer", "water", "cluster24", "chon60", "chon60s", "batch"),
                    default="chon60")
    ap.add_argument("--precision", choices=("f16x3", "mixed", "tf32x3", "fp64", "fp64tc"),
                    default="f16x3")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-batch", dest="with_batch", action="store_false",
                    help="leave out the 64-molecule batch record of the single-system runs")
    ap.add_argument("--batch-precision", choices=("f16x3", "mixed", "tf32x3", "fp64"), default="tf32x3",
                    help="the batch's precision, as a record of the single-system run and with "
                         "--workload batch (split TF32: its trial groups are at most 96 wide, "
                         "where the split-FP16 kernel is not the faster one)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch":
        gpu_batch_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
