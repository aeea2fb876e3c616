"""Benchmark: gate applications per second of the random-layer circuit.

Workload (one "step" = one pass of the whole hot path over one circuit):
  * state |0...0> initialised on the device (a1);
  * the 20-layer random-layer circuit -- U3(theta, phi, lambda) on every qubit,
    then CZ on (i, i+1) for even i in even layers and odd i in odd layers,
    angles ~ U[0, 2 pi) from seed 2 -- on n = 32 qubits in complex64 (32 GiB):
    950 gates, applied by the planner's tiled multi-gate passes (a2-a6);
  * read-out: squared norm and <sum_i Z_i Z_{i+1}> with FP64 accumulation (a8).
The state (32 GiB) is far larger than L2 (129 MB), so no L2 flush is needed.

Metric: logical (pre-fusion) gate applications per second, whole job (all
ranks). Multi-GPU: independent replicas, one per rank ("replicas only":
the single-state path does not shard without an exchange step), weak scaling.

``--impl reference`` times the CPU oracle (the plain complex128 unfused
simulator) on the host cores on a bounded sample of the same workload.

``--only NAME`` runs one secondary workload alone (variational_adjoint,
variational_adjoint_c128, adiabatic_batch, adiabatic_batch_c128, fused_tc,
unfused_passes, qft_n18_c128, random_layer_c128_n33, measurement,
host_memory, evolution, density_channels) and prints its result as one JSON line: for profiling those
kernels; it is not the benchmark line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gate apps/s (random-layer circuit, 20 layers)"
UNIT = "gate/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--qubits", dest="n", type=int, default=32)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--layers", type=int, default=20)
    ap.add_argument("--mode", default="auto", choices=["auto", "unfused", "tiled", "fused"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-jit", action="store_true",
                    help="run every tiled pass on the generic kernel (no specialised pass kernels)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workloads (variational adjoint)")
    ap.add_argument("--only", default=None, choices=sorted(SECONDARY),
                    help="run one secondary workload alone and print its result")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"random-layer circuit, {a.layers} layers, n={a.n}, {a.dtype}",
            "n_qubits": a.n, "state_dtype": a.dtype, "layers": a.layers, "seed": 2,
            "mode": a.mode, "state_bytes": (1 << a.n) * (8 if a.dtype == "c64" else 16),
            "l2_flush": "not needed: state larger than L2"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# GB300: 152 SMs x 128 FP32 lanes x 2 flops per FMA per clock. complex128
# passes compute in double-float on the same FP32 units.
SMS, FP32_LANES = 152, 128


def alu_peak_tflops(sm_mhz: float) -> float:
    return SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


TILED_SOURCES = ("kernels_tiled.cu", "tiled.h", "plan_tiled.cpp", "tile_device.cuh", "tile_jit.cpp", "device.cuh")
LAUNCH_PROFILE = os.path.join(ROOT, "profiles", "launches_random_layer_n32_c64.md")


def tiled_traffic(a):
    """DRAM bytes per launch of the tiled kernel from the committed ncu launch
    list, if it was taken on this workload from the current kernel sources
    (same source hash), else None."""
    import hashlib
    import re
    try:
        h = hashlib.sha256()
        for f in TILED_SOURCES:
            with open(os.path.join(ROOT, "paper_2009_01845_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        with open(LAUNCH_PROFILE) as fh:
            txt = fh.read()
        m = re.search(r"kernel sources sha256\[:16\][^:]*: ([0-9a-f]{16})", txt)
        b = re.search(r"tiled_kernel DRAM bytes per launch \(n = (\d+)\): (\d+)", txt)
        if m and b and m.group(1) == h.hexdigest()[:16] and int(b.group(1)) == a.n and a.dtype == "c64":
            return float(b.group(2))
    except OSError:
        pass
    return None


def roofline(name, rec, a, clk):
    """Roofline of the dominant kernel class. The bound is HBM bandwidth: the
    class's algorithmic bytes (one read and one write of the state per pass,
    B(n, b) = 2 * 2^n * b) over its CUDA-event time, against the measured copy
    bandwidth. A secondary ALU figure reports the same launches' arithmetic:
    flops are the implementation's own count of its rotation / diagonal-block
    decomposition (4 per amplitude per rotation, 12 per diagonal block, ...),
    and the peak is the FP32 unit count times the sampled SM clock (152 SMs x
    128 lanes x 2 flops per FMA). complex128 passes run in double-float on the
    same units: there the flops are the decomposition's count in complex128
    operations, each of which costs ~15-20 FP32 operations."""
    tot_ms, launches, nbytes, nflops = rec
    if not launches or tot_ms <= 0:
        return None
    bw, bw_src = measured_peaks()
    sm = clk.get("sm_mhz") or 2070.0
    alu = alu_peak_tflops(sm)
    t = tot_ms / 1000.0
    gbs = nbytes / t / 1e9
    tfl = nflops / t / 1e12
    return {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": bw, "unit": "GB/s", "frac": gbs / bw,
            "peak_source": f"{bw_src}: MEASURED_PEAKS hbm_gbs",
            "traffic": tiled_traffic(a) if name == "tiled" else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                              "profiles/launches_random_layer_n32_c64.md (null if the kernel sources changed)",
            "launches_per_step": launches / a.steps, "avg_launch_ms": tot_ms / launches,
            "bytes_per_launch": nbytes / launches,
            "alu": {"achieved": tfl, "peak": alu, "unit": "TFLOP/s", "frac": tfl / alu,
                    "flops_per_launch": nflops / launches,
                    "flops_source": "the implementation's own count of its decomposition" +
                                    ("" if a.dtype == "c64" else
                                     " (complex128 operations, each ~15-20 FP32 operations in double-float)"),
                    "peak_source": "FP32 units: 152 SMs x 128 lanes x 2 x median SM clock"}}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(a, budget_s: float = 12.0, threads: int = 1, n_s: int = 24):
    """Time the oracle (plain C complex128, unfused) on a bounded sample of the
    workload: the same circuit family at n_s qubits, first gates in order,
    until ~budget_s, with `threads` threads on the gate loop; per-gate time
    scaled by 2^(n - n_s) to the full n (gate cost is linear in 2^n)."""
    import oracle
    from paper_2009_01845_gb300 import inputs as qi
    n_s = min(a.n, n_s)
    used = oracle.set_threads(threads)
    gates = qi.random_layer_circuit(n_s, a.layers, seed=2)
    psi = oracle.zero_state(n_s)
    done, t0 = 0, time.perf_counter()
    for g in gates:
        oracle.apply_gate(psi, n_s, g)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    per_gate_full = dt / done * 2.0 ** (a.n - n_s)
    return {"value": 1.0 / per_gate_full, "unit": UNIT, "cores": used, "kind": "oracle",
            "extrapolated_from_n": n_s, "wall_s": dt,
            "sample": f"first {done} gates of the same circuit at n={n_s} (complex128, {used} thread(s), "
                      f"{dt:.1f} s), per-gate time scaled by 2^{a.n - n_s} to n={a.n}"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(a):
    """The oracle on all host cores (gate loop split by OpenMP), and on one
    core for reference; ~25 s of CPU work in total."""
    allc = oracle_sample(a, budget_s=12.0, threads=host_cores())
    one = oracle_sample(a, budget_s=8.0, threads=1)
    allc["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    return allc


def run_reference(a):
    """The reference arm: the oracle (the plain complex128 unfused simulator)
    on all host cores. A step is a bounded sample of the workload: the first
    gates of the same circuit at n = 24, whose per-gate time is scaled by
    2^(n - 24) to give the metric at the full n (labelled by
    extrapolated_from_n). ms_per_step is the sample's own wall time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    budget = max(2.0, 60.0 / max(1, a.steps + a.warmup))
    cores = host_cores()
    for i in range(a.warmup + a.steps):
        r = oracle_sample(a, budget_s=budget, threads=cores)
        if i >= a.warmup:
            per_step.append(r)
    v = statistics.median(x["value"] for x in per_step)
    ms = 1000.0 * statistics.mean(x["wall_s"] for x in per_step)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a), "extrapolated_from_n": per_step[-1]["extrapolated_from_n"],
            "step": "a bounded sample of the workload: the circuit's first gates at n=24, per-gate time "
                    "scaled by 2^(n-24); ms_per_step is that sample's wall time",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": per_step[-1]["cores"], "kind": "oracle",
                             "sample": per_step[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ secondary workloads
def specialise(fn, fold: bool = False):
    """Run fn once with every new tiled pass structure queued for a
    specialised kernel, wait for the compiles, and go back to the default
    policy: later runs of passes of those structures use the specialised
    kernels. fold: run it a second time, which queues kernels with the passes'
    values compiled in as well (for a circuit that repeats with fixed angles)."""
    from paper_2009_01845_gb300 import qsim
    qsim.jit_set_policy("eager", fold=fold)
    try:
        fn()
        qsim.jit_wait()
        if fold:
            fn()
            qsim.jit_wait()
    finally:
        qsim.jit_set_policy("tiered")


def _time_cuda(fn, steps: int, warmup: int = 2, jit: bool = True) -> float:
    """Mean ms of fn() over `steps` calls, CUDA events on the current stream;
    the warm-up specialises fn's tiled passes first unless jit is False."""
    import torch
    if jit and warmup > 0:
        specialise(fn)
        warmup -= 1
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def variational_adjoint(steps: int = 5, dtype: str = "c64") -> dict:
    """Variational ansatz n = 20, 10 layers of RY + CZ ladder, 256 parameter sets
    (seed 4), complex64 (complex128: the same in double-float), TFIM energy
    g = 1: forward (incl. lambda = H psi and the energy) vs forward + adjoint
    reverse sweep, through qs_energy_gradient."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    n, L, B = 20, 10, 256
    th = qi.variational_params(B, L, n, seed=4)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qsim.param_indices(tmpl)
    eng = qsim.EnergyGradient(n, B, tmpl, pidx, qi.tfim_terms(n, 1.0), dtype=dtype)
    params = torch.tensor(th.reshape(B, -1), device="cuda")
    energy = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty(B, P, dtype=torch.float64, device="cuda")
    t_fwd = _time_cuda(lambda: eng.run(params, mode="forward", energy=energy), steps)
    t_full = _time_cuda(lambda: eng.run(params, mode="full", energy=energy, grad=grad), steps)
    qsim.profile_collect()
    qsim.profile_enable(True)
    eng.run(params, mode="full", energy=energy, grad=grad)
    torch.cuda.synchronize()
    qsim.profile_enable(False)
    prof = qsim.profile_collect()
    t_hpsi = prof.get("hpsi", (0.0,))[0]
    return {"workload": f"variational n=20, 10 layers, batch 256, {dtype}, TFIM g=1",
            "forward_ms": t_fwd, "forward_plus_adjoint_ms": t_full, "hpsi_ms": t_hpsi,
            # the reverse sweep plus lambda = H psi, over the forward without it
            "adjoint_incl_hpsi_over_forward": (t_full - t_fwd + t_hpsi) / (t_fwd - t_hpsi),
            # the reverse sweep including H psi over the forward including the
            # energy (which needs H psi too)
            "sweep_incl_hpsi_over_forward_incl_energy": (t_full - t_fwd + t_hpsi) / t_fwd,
            "adjoint_over_forward": (t_full - t_fwd) / t_fwd, "total_over_forward": t_full / t_fwd,
            "gradients_per_s": B * P / (t_full / 1000.0),
            "kernels_full_call": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}}


def adiabatic_batch(steps: int = 100, dtype: str = "c64") -> dict:
    """Adiabatic evolution batch: 64 instances, n ~ U{16..26} (seed 5), H0 = -sum X,
    H1 = sum J_ij Z_i Z_j + sum h_i Z_i with J, h ~ N(0, 1), linear schedule,
    T = 10, dt = 0.01, |+>^n. Timed on the first `steps` of the 1000 steps
    (each step costs the same): all widths in one call, side by side on streams
    of their own ("one_call"), one batched call per width in turn ("batched"),
    and instance by instance ("sequential"). Reports instance-steps/s;
    also the final energy and the ground-state overlap of the smallest
    instance after all 1000 steps (ground state by brute force over 2^16)."""
    import numpy as np
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    inst = qi.adiabatic_instances(64, seed=5)
    T, dt = 10.0, 0.01
    widths = sorted({m for m, _, _ in inst})
    groups = {w: [i for i, (m, _, _) in enumerate(inst) if m == w] for w in widths}
    states = {w: qsim.State(w, batch=len(ix), dtype=dtype) for w, ix in groups.items()}

    def batched():
        for w, ix in groups.items():
            states[w].init_plus().adiabatic_evolve_batch(inst[ix[0]][1], [inst[i][2] for i in ix], T, dt,
                                                         steps=steps)

    t_b = _time_cuda(batched, 1, warmup=1)
    # every width in one call: the handles evolve side by side on their own streams
    h0s = [inst[groups[w][0]][1] for w in widths]
    h1s = [inst[i][2] for w in widths for i in groups[w]]
    order = [states[w] for w in widths]

    def one_call():
        for st_ in order:
            st_.init_plus()
        qsim.adiabatic_run_batch(order, h0s, h1s, T, dt, steps=steps)

    t_o = _time_cuda(one_call, 1, warmup=1)
    # device time by kernel class of one batched run (the rest of t_b is host work)
    qsim.profile_collect()
    qsim.profile_enable(True)
    batched()
    torch.cuda.synchronize()
    qsim.profile_enable(False)
    prof_raw = qsim.profile_collect()
    prof_b = {k: {"ms": v[0], "launches": v[1], "GB": v[2] / 1e9} for k, v in prof_raw.items() if v[1]}
    # algorithmic bytes: every tiled pass reads and writes its members' states once
    alg_bytes = sum(v[2] for v in prof_raw.values())
    bw, _ = measured_peaks()
    solo = {w: qsim.State(w, dtype=dtype) for w in widths}

    def sequential():
        for m, h0, h1 in inst:
            solo[m].init_plus().adiabatic_evolve(h0, h1, T, dt, steps=steps)

    t_s = _time_cuda(sequential, 1, warmup=1)
    # the smallest instance, all 1000 steps: energy and ground-state overlap
    m0, h0, h1 = inst[min(groups[widths[0]])]
    st = qsim.State(m0, dtype=dtype).init_plus().adiabatic_evolve(h0, h1, T, dt)
    e_final = float(st.expectation(h1)[0].real)
    idx = np.arange(1 << m0)
    E = np.zeros(1 << m0)
    for c, _, zm in h1:
        par = np.zeros(1 << m0, dtype=np.int64)
        for q in range(m0):
            if (zm >> q) & 1:
                par ^= (idx >> (m0 - 1 - q)) & 1
        E += c * (1 - 2 * par)
    gmin = E.min()
    ground = np.flatnonzero(np.isclose(E, gmin, rtol=0, atol=1e-12))
    p = st.probabilities()
    del states, solo
    torch.cuda.empty_cache()
    isteps = 64 * steps
    return {"workload": f"adiabatic batch: 64 instances n in [16,26] (seed 5), T=10, dt=0.01, {dtype}, "
                        f"first {steps} of 1000 second-order Trotter steps timed",
            "one_call_ms": t_o, "batched_ms": t_b, "sequential_ms": t_s,
            "instance_steps_per_s_one_call": isteps / (t_o / 1000.0),
            "one_call_hbm_frac": alg_bytes / (t_o / 1000.0) / 1e9 / bw,
            "instance_steps_per_s_batched": isteps / (t_b / 1000.0),
            "instance_steps_per_s_sequential": isteps / (t_s / 1000.0),
            "projected_full_run_s_batched": t_b / 1000.0 * 1000 / steps,
            "algorithmic_GB_per_step": alg_bytes / steps / 1e9,
            "batched_hbm_frac": alg_bytes / (t_b / 1000.0) / 1e9 / bw,
            "tiled_hbm_frac": (prof_raw["tiled"][2] / (prof_raw["tiled"][0] / 1000.0) / 1e9 / bw
                               if prof_raw.get("tiled", (0,))[0] else None),
            "kernels_batched_run": prof_b,
            "widths": {int(w): len(ix) for w, ix in groups.items()},
            "smallest_instance": {"n": m0, "final_energy": e_final, "ground_energy": float(gmin),
                                  "ground_state_overlap": float(p[ground].sum())}}


def fused_tc(steps: int = 2) -> dict:
    """Random-layer circuit (20 layers, seed 3) at n = 30 in complex64: gates fused
    into 5-qubit blocks applied as 3xTF32 tensor-core contractions, against the
    tiled CUDA-core passes on the same state."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    n = 30
    gates = qi.random_layer_circuit(n, 20, seed=3)
    st = qsim.State(n, dtype="c64")
    out = {}
    for mode in ("fused", "tiled"):
        t = _time_cuda(lambda: st.init_basis(0).apply(gates, mode=mode), steps, warmup=1)
        qsim.profile_collect()
        qsim.profile_enable(True)
        st.init_basis(0).apply(gates, mode=mode)
        torch.cuda.synchronize()
        qsim.profile_enable(False)
        prof = qsim.profile_collect()
        key = "fused_tc" if mode == "fused" else "tiled"
        ms, launches, nbytes, nflops = prof[key]
        out[mode] = {"ms_per_circuit": t, "gate_apps_per_s": len(gates) / (t / 1000.0),
                     "passes": launches, "avg_pass_ms": ms / max(1, launches),
                     "hbm_GBps": nbytes / (ms / 1000.0) / 1e9 if ms else None,
                     "TFLOPs_algorithmic": nflops / (ms / 1000.0) / 1e12 if ms else None}
    # error of the fused result against the complex128 tiled path on the same GPU
    st.init_basis(0).apply(gates, mode="fused")
    ref = qsim.State(n, dtype="c128").init_basis(0).apply(gates, mode="tiled")
    torch.cuda.synchronize()
    diff = st.tensor.to(torch.complex128) - ref.tensor
    out["fused_error_vs_c128"] = {"max_abs": float(diff.abs().max()), "l2": float(torch.linalg.vector_norm(diff))}
    del diff
    st.init_basis(0).apply(gates, mode="tiled")
    torch.cuda.synchronize()
    diff = st.tensor.to(torch.complex128) - ref.tensor
    out["tiled_error_vs_c128"] = {"max_abs": float(diff.abs().max()), "l2": float(torch.linalg.vector_norm(diff))}
    del diff
    ref.close()
    del ref
    st.close()
    del st
    torch.cuda.empty_cache()
    out["workload"] = "random-layer circuit, 20 layers, seed 3, n=30, complex64 (error against complex128 tiled)"
    return out


def _peak_hbm() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def unfused_passes(n: int = 32, reps: int = 5) -> dict:
    """One-gate passes (the plain unfused simulator) at n = 32: a dense 1-qubit
    gate on the lowest and the highest index bit, a 2-qubit dense gate, CZ and
    SWAP in complex64, and the dense 1- and 2-qubit gates in complex128 (in
    double-float and in FP64 arithmetic); per pass the
    CUDA-event time, the algorithmic bytes (2^n reads and writes of the
    amplitudes the gate touches) and the fraction of the measured HBM peak."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    G = qi.Gate
    u4 = qi.random_unitary(2, qi.rng(7))
    cases = [("c64", "H on qubit n-1 (index bit 0)", G("H", (n - 1,))),
             ("c64", "H on qubit 0 (index bit n-1)", G("H", (0,))),
             ("c64", "U3 on qubit n/2", G("U3", (n // 2,), (), (0.3, 0.2, 0.1))),
             ("c64", "dense 2-qubit on qubits (3, n-5)", G("UNITARY", (3, n - 5), (), (), u4)),
             ("c64", "CZ(0, 1)", G("CZ", (0, 1))),
             ("c64", "SWAP(2, n-3)", G("SWAP", (2, n - 3))),
             ("c128", "H on qubit n-1 (index bit 0)", G("H", (n - 1,))),
             ("c128", "U3 on qubit n/2", G("U3", (n // 2,), (), (0.3, 0.2, 0.1))),
             ("c128", "dense 2-qubit on qubits (3, n-5)", G("UNITARY", (3, n - 5), (), (), u4))]
    peak = _peak_hbm()
    out = {"workload": f"one-gate passes, n={n}", "peak_hbm_GBps": peak, "passes": []}
    st = None
    cur = None
    for dt, name, g in cases:
        if dt != cur:
            if st is not None:
                st.close()
                del st
                torch.cuda.empty_cache()
            st = qsim.State(n, dtype=dt).init_plus()
            cur = dt
        # complex128: the default double-float arithmetic and the FP64 one
        for fp64 in ((False, True) if dt == "c128" else (False,)):
            t = _time_cuda(lambda: st.apply([g], mode="unfused", fp64=fp64), reps, warmup=2)
            qsim.profile_collect()
            qsim.profile_enable(True)
            st.apply([g], mode="unfused", fp64=fp64)
            torch.cuda.synchronize()
            qsim.profile_enable(False)
            prof = qsim.profile_collect()
            nbytes = sum(v[2] for v in prof.values())
            gbs = nbytes / (t / 1000.0) / 1e9
            rec = {"dtype": dt, "gate": name, "ms": t, "GB": nbytes / 1e9, "GBps": gbs,
                   "frac_of_measured_hbm": gbs / peak}
            if dt == "c128":
                rec["arithmetic"] = "fp64" if fp64 else "double-float"
            out["passes"].append(rec)
    if st is not None:
        st.close()
        del st
        torch.cuda.empty_cache()
    return out


def qft_n18(reps: int = 20) -> dict:
    """QFT on n = 18 qubits in complex128 (4 MiB: the state stays in L2), input
    a seeded basis state: per-call time of the 180-gate circuit one gate per
    pass (the plain method), in tiled passes, and replayed from a CUDA-graph
    plan of the unfused passes (no host launch overhead); max error against the
    closed form 2^{-n/2} exp(2 pi i x k / 2^n)."""
    import numpy as np
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    n = 18
    x = qi.qft_input(n, seed=1)
    gates = qi.qft_circuit(n)
    st = qsim.State(n, dtype="c128")
    out = {"workload": f"QFT n={n} complex128, |x> with x = {x} (seed 1), {len(gates)} gates"}
    for mode in ("unfused", "tiled"):
        t = _time_cuda(lambda: st.init_basis(x).apply(gates, mode=mode), reps, warmup=2)
        out[mode] = {"ms_per_circuit": t, "gate_apps_per_s": len(gates) / (t / 1000.0)}
    k = np.arange(1 << n)
    want = np.exp(2j * np.pi * x * k / (1 << n)) / np.sqrt(1 << n)
    for mode in ("unfused", "tiled"):
        plan = qsim.Plan(st, gates, mode=mode, autotune=False)
        t = _time_cuda(lambda: (st.init_basis(x), plan.execute()), reps, warmup=2)
        st.init_basis(x)
        plan.execute()
        out[mode + "_graph"] = {"ms_per_circuit": t, "gate_apps_per_s": len(gates) / (t / 1000.0),
                                "graph_nodes": plan.info()["graph_nodes"],
                                "max_abs_error_vs_closed_form": float(np.max(np.abs(st.get() - want)))}
        plan.close()
    st.close()
    del st
    torch.cuda.empty_cache()
    return out


def random_layer_c128(n: int = 33, layers: int = 2) -> dict:
    """The whole 20-layer random-layer circuit (seed 2) at n = 33 in complex128
    (128 GiB state) in tiled passes, double-float arithmetic on specialised
    kernels, timed end to end (one run after a run that specialises its
    passes); then its first `layers` layers in tiled FP64 passes and in the
    plain unfused simulator (double-float and FP64), with the full-circuit
    times their per-gate rates project."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    full = qi.random_layer_circuit(n, 20, seed=2)
    part = qi.random_layer_circuit(n, layers, seed=2)
    st = qsim.State(n, dtype="c128")
    out = {"workload": f"random-layer circuit, 20 layers ({len(full)} gates), n={n}, complex128"}
    t = _time_cuda(lambda: st.init_basis(0).apply(full, mode="tiled"), 1, warmup=1)
    qsim.profile_collect()
    qsim.profile_enable(True)
    st.init_basis(0).apply(full, mode="tiled")
    torch.cuda.synchronize()
    qsim.profile_enable(False)
    ms, launches, nbytes, _ = qsim.profile_collect()["tiled"]
    out["tiled"] = {"ms": t, "gate_apps_per_s": len(full) / (t / 1000.0), "gates": len(full),
                    "arithmetic": "double-float", "kernels": "specialised", "passes": launches,
                    "avg_pass_ms": ms / max(1, launches),
                    "pass_hbm_frac": nbytes / (ms / 1000.0) / 1e9 / _peak_hbm() if ms else None}
    out["norm2_after"] = float(st.norm2()[0])
    for mode, fp64, key in (("tiled", True, "tiled_fp64"), ("unfused", False, "unfused"),
                            ("unfused", True, "unfused_fp64")):
        st.init_basis(0)
        torch.cuda.synchronize()
        t = _time_cuda(lambda: st.apply(part, mode=mode, fp64=fp64), 1, warmup=0)
        rate = len(part) / (t / 1000.0)
        out[key] = {"ms": t, "gate_apps_per_s": rate, "gates": len(part),
                    "arithmetic": "fp64" if fp64 else "double-float",
                    "projected_full_circuit_s": len(full) / rate}
    st.close()
    del st
    torch.cuda.empty_cache()
    return out


def _profiled(fn):
    """Run fn once with the library's per-class launch accounting on: class ->
    (ms, launches, GB, GB/s as a fraction of the measured HBM peak)."""
    import torch
    from paper_2009_01845_gb300 import qsim
    qsim.profile_collect()
    qsim.profile_enable(True)
    fn()
    torch.cuda.synchronize()
    qsim.profile_enable(False)
    peak = _peak_hbm()
    out = {}
    for k, v in qsim.profile_collect().items():
        ms, launches, nbytes = v[0], v[1], v[2]
        if launches:
            out[k] = {"ms": ms, "launches": launches, "GB": nbytes / 1e9,
                      "hbm_frac": nbytes / (ms / 1000.0) / 1e9 / peak if ms > 0 and nbytes else None}
    return out


def evolution(n: int = 24, steps: int = 10) -> dict:
    """Exact time evolution (Sec. 2.6) at n = 24: H(s) = (1 - s) H0 + s H1,
    H0 = -sum X, H1 = a seeded Ising chain with fields plus 8 random Pauli
    terms; T = steps * dt, dt = 0.05; the exp (Taylor), rk4 and rk45 solvers
    in complex64 and complex128: steps/s and the kernels' HBM fractions
    (H psi and the state combinations)."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(31)) + qi.random_pauli_terms(n, 8, seed=32)
    dt = 0.05
    out = {"workload": f"exact evolution, n={n}, {steps} steps of dt={dt}, H0 = -sum X, H1 = Ising + 8 Pauli terms"}
    for dtype in ("c64", "c128"):
        st = qsim.State(n, dtype=dtype)
        for solver in ("exp", "rk4", "rk45"):
            run = lambda: st.init_plus().evolve(h0, h1, steps * dt, dt, solver=solver)
            t = _time_cuda(run, 1, warmup=1, jit=False)
            out[f"{dtype}_{solver}"] = {"ms": t, "steps_per_s": steps / (t / 1000.0), "kernels": _profiled(run)}
        st.close()
        del st
        torch.cuda.empty_cache()
    return out


def density_channels(n: int = 14, layers: int = 4) -> dict:
    """Density matrices and noise (Sec. 2.4) at n = 14 (rho as a 28-qubit
    vector): per layer U3 on every qubit and the CZ ladder (random-layer
    circuit, seed 6) as rho -> U rho U^dag, then a depolarizing channel
    (p = 0.01) on every qubit, in complex64 and complex128: gates and channels
    per second and the kernels' HBM fractions."""
    import numpy as np
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    gates = qi.random_layer_circuit(n, layers, seed=6)
    p = 0.01
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    dep = [np.sqrt(1 - 3 * p / 4) * np.eye(2), np.sqrt(p / 4) * X, np.sqrt(p / 4) * Y, np.sqrt(p / 4) * Z]
    chans = [([q], dep) for q in range(n)]
    per_layer = len(gates) // layers
    out = {"workload": f"density matrix n={n} (4^n entries), {layers} random layers + depolarizing p={p} on every qubit"}
    for dtype in ("c64", "c128"):
        dm = qsim.DensityMatrix(n, dtype=dtype)
        psi0 = np.zeros(1 << n, dtype=complex)
        psi0[0] = 1.0

        def run():
            dm.init_pure(psi0)
            for l in range(layers):
                dm.apply(gates[l * per_layer:(l + 1) * per_layer])
                dm.apply_channels(chans)

        t = _time_cuda(run, 1, warmup=2)
        ops = len(gates) + layers * n
        out[dtype] = {"ms": t, "ops_per_s": ops / (t / 1000.0), "trace": float(dm.trace()[0]),
                      "kernels": _profiled(run)}
        del dm
        torch.cuda.empty_cache()
    return out


def summary(line: dict) -> dict:
    """A compact digest of the line: headline, roofline, and one or two
    figures per secondary workload."""
    def get(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def rnd(x, k=4):
        return None if x is None else float(f"{x:.{k}g}")

    sec = line.get("secondary", {})
    out = {"gate_per_s": rnd(line["value"]), "ms_per_step": rnd(line["ms_per_step"]),
           "pass_kernels": get(line, "pass_kernels", "timed_region"),
           "tiled_hbm_frac": rnd(get(line, "roofline", "frac"), 3),
           "tiled_alu_frac": rnd(get(line, "roofline", "alu", "frac"), 3),
           "e2e_gate_per_s": rnd(get(line, "e2e", "value")),
           "cpu_gate_per_s": rnd(get(line, "cpu_baseline", "value")),
           "cpu_cores": get(line, "cpu_baseline", "cores")}
    va = sec.get("variational_adjoint_c128")
    if va:
        out["adjoint_c128"] = {"fwd_ms": rnd(va["forward_ms"]), "full_ms": rnd(va["forward_plus_adjoint_ms"]),
                               "total_over_fwd": rnd(va["total_over_forward"], 3)}
    va = sec.get("variational_adjoint")
    if va:
        out["adjoint"] = {"fwd_ms": rnd(va["forward_ms"]), "full_ms": rnd(va["forward_plus_adjoint_ms"]),
                          "adj_incl_hpsi_over_fwd": rnd(va["adjoint_incl_hpsi_over_forward"], 3),
                          "sweep_incl_hpsi_over_fwd_incl_energy":
                              rnd(va.get("sweep_incl_hpsi_over_forward_incl_energy"), 3),
                          "total_over_fwd": rnd(va["total_over_forward"], 3)}
    for key, name in (("adiabatic_batch", "adiabatic"), ("adiabatic_batch_c128", "adiabatic_c128")):
        ab = sec.get(key)
        if ab:
            out[name] = {k: rnd(v) for k, v in ab.items() if k.startswith("instance_steps") or
                         k.endswith("hbm_frac")}
    ft = sec.get("fused_tc")
    if ft:
        out["fused_tc"] = {"fused_gate_per_s": rnd(get(ft, "fused", "gate_apps_per_s")),
                           "tiled_gate_per_s": rnd(get(ft, "tiled", "gate_apps_per_s")),
                           "fused_pass_ms": rnd(get(ft, "fused", "avg_pass_ms"))}
    up = sec.get("unfused_passes")
    if up:
        out["unfused_hbm_frac"] = {" ".join([p["dtype"], p["gate"]] + ([p["arithmetic"]] if "arithmetic" in p else [])):
                                   rnd(p["frac_of_measured_hbm"], 3) for p in up["passes"]}
    q = sec.get("qft_n18_c128")
    if q:
        out["qft_n18_gate_per_s"] = {k: rnd(v["gate_apps_per_s"]) for k, v in q.items() if isinstance(v, dict)}
    rc = sec.get("random_layer_c128_n33")
    if rc:
        out["c128_n33_gate_per_s"] = {k: rnd(v["gate_apps_per_s"]) for k, v in rc.items() if isinstance(v, dict)}
        out["c128_n33_full_circuit_s"] = rnd(get(rc, "tiled", "ms") / 1000.0) if get(rc, "tiled", "ms") else None
    ev = sec.get("evolution")
    if ev:
        out["evolution_steps_per_s"] = {k: rnd(v["steps_per_s"]) for k, v in ev.items() if isinstance(v, dict)}
    dc = sec.get("density_channels")
    if dc:
        out["density_ops_per_s"] = {k: rnd(v["ops_per_s"]) for k, v in dc.items() if isinstance(v, dict)}
    ms = sec.get("measurement")
    if ms:
        out["marginal_hbm_frac"] = [rnd(m["frac_of_measured_hbm"], 3) for m in ms["marginals"]]
    return out


# ------------------------------------------------------------------ multi-rank helpers
def max_over_ranks(x: float, world: int) -> float:
    """The maximum of x over all ranks (the slowest replica sets the job's
    time); x itself at world size 1. Uses the process group's backend (a CUDA
    tensor for NCCL, a CPU tensor for gloo)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, gates_per_step: int, ms_per_step: float) -> float:
    """Gate applications per second of the whole job: every replica applies the
    step's gates once per step (weak scaling), timed by the slowest replica."""
    return world * gates_per_step / (ms_per_step / 1000.0)


# ------------------------------------------------------------------ GPU arm
def run_ours(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2009_01845_gb300 import build as qbuild
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim

    if rank == 0 or not os.path.exists(qbuild.LIB):
        qbuild.build()
    barrier()
    qsim.load()

    n = a.n
    gates = qi.random_layer_circuit(n, a.layers, seed=2)
    zz = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    st = qsim.State(n, dtype=a.dtype)
    gate_arr, keep = qsim.marshal_gates(gates)
    o = qsim.opts(a.mode)
    zz_arr, zz_n = qsim.marshal_terms(zz)
    import ctypes
    import numpy as np
    out_re = np.zeros(1)
    out_n = np.zeros(1)

    def step():
        st.init_basis(0)
        qsim._check(st.lib.qs_apply_gates(st.handle, gate_arr, len(gates), ctypes.byref(o)))
        qsim._check(st.lib.qs_norm2(st.handle, ctypes.c_void_p(out_n.ctypes.data)))
        qsim._check(st.lib.qs_expectation(st.handle, zz_arr, zz_n, ctypes.c_void_p(out_re.ctypes.data), None))

    # warm-up: the first step queues a specialised kernel for every tiled pass
    # and waits for the compiles; the rest run as the timed steps do
    if a.no_jit:
        qsim.jit_set_policy("off")
    for i in range(a.warmup):
        if i == 0 and not a.no_jit:
            specialise(step, fold=True)  # the step repeats one circuit with fixed angles
        else:
            step()
    torch.cuda.synchronize()
    jit_after_warmup = qsim.jit_stats()
    if abs(out_n[0] - 1.0) > 1e-3:
        raise RuntimeError(f"norm drifted: {out_n[0]}")

    clocks = ClockSampler(local)
    qsim.profile_collect()
    qsim.profile_enable(True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for _ in range(a.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    qsim.profile_enable(False)
    prof = qsim.profile_collect()
    jit_timed = {k: v - jit_after_warmup[k] for k, v in qsim.jit_stats().items()
                 if k in ("specialised_launches", "generic_launches")}
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, world)
    value = whole_job_value(world, len(gates), ms)

    # roofline of the dominant kernel class: algorithmic bytes and flops tallied
    # by the library per launch, over the CUDA-event time of those launches
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    roof = roofline(dom[0], dom[1], a, clk)
    launches_total = int(sum(v[1] for v in prof.values()))

    # end to end through the public Python API with host inputs: marshal the
    # gate list from Python objects, apply, read back the results to the host
    e2e = None
    if not a.no_e2e:
        e_steps = max(1, min(a.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(e_steps):
            st.init_basis(0)
            arr, kp = qsim.marshal_gates(gates)
            h2d = ctypes.sizeof(arr) + 8
            qsim._check(st.lib.qs_apply_gates(st.handle, arr, len(gates), ctypes.byref(o)))
            r1 = st.norm2()
            r2 = st.expectation(zz)
            d2h = r1.nbytes + 16
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1000.0 / e_steps
        e2e = {"value": world * len(gates) / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a)
    secondary = {}
    if not a.no_secondary:
        st.close()
        del st
        torch.cuda.empty_cache()
        for name, fn in SECONDARY.items():
            secondary[name] = fn()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if a.dtype == "c64" else "f64",
                "data": "synthetic", "config": workload_config(a),
                "parallelism": "replicas" if world > 1 else "single",
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_total,
                "kernels": {k: {"ms_per_step": v[0] / a.steps, "launches_per_step": v[1] / a.steps,
                                "GB_per_step": v[2] / a.steps / 1e9, "GFLOP_per_step": v[3] / a.steps / 1e9}
                            for k, v in prof.items() if v[1]},
                "energy_zz": float(out_re[0]), "norm2": float(out_n[0]),
                "pass_kernels": {"timed_region": jit_timed,
                                 "compiled": jit_after_warmup["compiled"],
                                 "compile_seconds": jit_after_warmup["compile_seconds"],
                                 "failed": jit_after_warmup["failed"]},
                "secondary": secondary}
        # the key figures once more, last, so that a truncated log keeps them
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if a.no_secondary:
        st.close()
    if world > 1:
        dist.destroy_process_group()


def measurement(n: int = 32, reps: int = 3) -> dict:
    """Measurement simulation (Sec. 3.3): H on every qubit at n = 32 complex64
    (the paper's sampling benchmark), then samples of all qubits for 10^3 ..
    10^7 device-side uniforms (seed 13), and the outcome probabilities of a
    12-qubit and a 1-qubit group; CUDA-event times, median of `reps`, state
    preparation excluded (as the paper subtracts it). A sampling call reads the
    state once for its block sums, then each shot scans part of one block."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    st = qsim.State(n, dtype="c64").init_basis(0)
    st.apply([qi.Gate("H", (q,)) for q in range(n)], mode="tiled")
    torch.cuda.synchronize()
    bw, _ = measured_peaks()
    state_gb = (1 << n) * 8 / 1e9

    def med(fn):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"workload": f"H on every qubit, n={n}, complex64; samples of all qubits; group marginals",
           "sampling": [], "marginals": []}
    g = torch.Generator(device="cuda").manual_seed(13)
    for shots in (10 ** 3, 10 ** 5, 10 ** 6, 10 ** 7):
        u = torch.rand(shots, dtype=torch.float64, device="cuda", generator=g)
        st.sample(u)  # warm-up
        ms = med(lambda: st.sample(u))
        out["sampling"].append({"shots": shots, "ms": ms, "shots_per_s": shots / (ms / 1000.0)})
    for grp in (list(range(12)), [n - 1]):
        st.marginal_probabilities(grp)
        ms = med(lambda: st.marginal_probabilities(grp))
        out["marginals"].append({"qubits": len(grp), "ms": ms, "GBps": state_gb / (ms / 1000.0),
                                 "frac_of_measured_hbm": state_gb / (ms / 1000.0) / bw})
    st.close()
    torch.cuda.empty_cache()
    return out


def host_memory(n: int = 34, layers: int = 2, device_gib: int = 16) -> dict:
    """A state in host memory (Sec. 2.5: one device reused for a state's
    pieces): the random-layer circuit's first layers at n = 34 complex64
    (128 GiB of pinned host memory, the largest power of two the host holds)
    through a device budget of 16 GiB; per-gate rate and the achieved
    host<->device (C2C) bandwidth: every segment copies the state to the
    device and back once."""
    import torch
    from paper_2009_01845_gb300 import inputs as qi
    from paper_2009_01845_gb300 import qsim
    gates = qi.random_layer_circuit(n, layers, seed=2)
    t0 = time.perf_counter()
    hs = qsim.HostState(n, dtype="c64", device_bytes=device_gib << 30)
    t_alloc = time.perf_counter() - t0
    hs.init_basis(0)
    qsim.profile_collect()
    qsim.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs.apply(gates)
    nrm = hs.norm2()[0]  # synchronises
    t = time.perf_counter() - t0
    qsim.profile_enable(False)
    raw = qsim.profile_collect()
    state = (1 << n) * 8
    hs.close()
    hc = raw.get("host_copy", (0.0, 0, 0.0, 0.0))
    return {"workload": f"random-layer circuit, first {layers} layers, n={n}, complex64, state in host memory, "
                        f"device budget {device_gib} GiB", "gates": len(gates), "wall_s": t,
            "gate_apps_per_s": len(gates) / t, "host_alloc_s": t_alloc, "norm2": nrm,
            "state_GiB": state / 2 ** 30,
            "host_copy_GB": hc[2] / 1e9, "host_copy_GBps": hc[2] / (hc[0] / 1000.0) / 1e9 if hc[0] else None,
            "state_passes_over_c2c": hc[2] / (2 * state) if state else None,
            "kernels": {k: {"ms": v[0], "launches": v[1], "GB": v[2] / 1e9} for k, v in raw.items() if v[1]},
            "note": "wall time includes the final norm pass (one more stream of the state)"}


SECONDARY = {
    "variational_adjoint": lambda: variational_adjoint(),
    "variational_adjoint_c128": lambda: variational_adjoint(steps=2, dtype="c128"),
    "adiabatic_batch": lambda: adiabatic_batch(),
    "adiabatic_batch_c128": lambda: adiabatic_batch(steps=50, dtype="c128"),
    "fused_tc": lambda: fused_tc(),
    "unfused_passes": lambda n=32: unfused_passes(n=n),
    "qft_n18_c128": lambda: qft_n18(),
    "random_layer_c128_n33": lambda: random_layer_c128(),
    "measurement": lambda: measurement(),
    "evolution": lambda: evolution(),
    "density_channels": lambda: density_channels(),
    "host_memory": lambda: host_memory(),
}


def main():
    a = parse()
    if a.only:
        # --n sizes the one-gate passes (e.g. a small case for a profiler)
        fn = SECONDARY[a.only]
        res = fn(n=a.n) if a.only == "unfused_passes" else fn()
        print(json.dumps({a.only: res}), flush=True)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
