#!/usr/bin/env python
"""Throughput of the SSP-RK3 pseudo-spectral step on GB300.

Metric: grid-point steps per second, sum over members of N^3 x completed RK3
steps / second (one step = three evaluations of Algorithm 2 + the RK3
combines).  Default workload: one 256^3 sample per GPU in FP32 (padded grid
384^3), seeded random divergence-free initial data with E(k) ~ k^4
exp(-2 (k/4)^2) and energy 0.5, the hyper-viscosity for N (s = 1.5,
theta = 1/2, eps0 = m_N coefficient = 1), CFL 0.5.  Inputs live in HBM when
the timed region starts; every step streams about 18 GB, far above the
126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank advances its own sample (weak scaling: the Monte
Carlo ensemble shards with no data-path collective).  Rank 0 prints one JSON
line.  ``--impl reference`` times the CPU oracle instead (the paper has no
code to run): each step is one RK3 step of the oracle at 16^3, a bounded
sample of the workload labelled as such in its config.
"""
from __future__ import annotations

import argparse
import math
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

METRIC = "grid-pt-steps/s at 256^3 (plain vs batched FP32 ensemble), % of HBM roofline"
UNIT = "grid-pt-steps/s"


ENSEMBLE_LEVELS = [(64, 256, 1000), (128, 32, 2000), (256, 4, 3000)]   # (N, members, seed base)


def _ic(args):
    N, seed, member = args
    import ns3d_inputs as I
    return I.random_spectrum(N, seed=seed, member=member)


def ensemble_ics(levels):
    """Seeded initial data of every member, built in a spawn-started pool."""
    import multiprocessing as mp
    jobs = [(N, base, m) for N, M, base in levels for m in range(M)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        return pool.map(_ic, jobs, chunksize=4)


def bench_ensemble(B, torch, steps: int, warmup: int, to_t: float = 0.0):
    """Batched uneven FP32 ensemble: 256 x 64^3 + 32 x 128^3 + 4 x 256^3 members
    in one plan (one level per resolution), per-member CFL steps."""
    Ns = [N for N, M, _ in ENSEMBLE_LEVELS for _ in range(M)]
    ics = ensemble_ics(ENSEMBLE_LEVELS)
    plan = B.Plan(Ns, B.NS3D_F32, eps0=1.0, cfl=0.5)
    for m, u in enumerate(ics):
        plan.set_initial(m, u)
    del ics
    stream = torch.cuda.current_stream()
    plan.step(warmup, t_end=to_t)
    plan.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.step(steps, t_end=to_t)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pts = sum(N ** 3 for N in Ns)
    # byte model per level: the four passes of a fused FP32 level (inverse y,
    # z, forward y, fused x), each member's arrays read and written once per
    # pass and stage; no reuse through L2 is assumed (the 64^3 level's 256
    # members hold ~7.7 GB of arrays, far above the 126 MB L2)
    peak, peak_kind = measured_peaks()
    levels, step_bytes = {}, 0.0
    first = 0
    for N, M, _ in ENSEMBLE_LEVELS:
        P = plan.info(first)["P"]
        kb = kernel_bytes(N, P, 8, M)
        b = 3 * sum(kb[k] for k in ("inverse_y", "zpass", "forward_y", "fused_x"))
        levels[str(N)] = {"members": M, "P": P, "bytes_per_step": b}
        step_bytes += b
        first += M
    ach = step_bytes / (ms / steps * 1e-3) / 1e9
    info = {"members": {str(N): M for N, M, _ in ENSEMBLE_LEVELS}, "steps": steps,
            "ms_per_step": ms / steps, "value": pts * steps / (ms * 1e-3), "unit": UNIT,
            "samples_steps_per_s": len(Ns) * steps / (ms * 1e-3),
            "gpu_launches_per_step": plan.info(0)["launches_per_step"],
            "roofline": {"bound": "hbm", "bytes_per_step": step_bytes, "achieved": ach,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                         "levels": levels}}
    if to_t > 0:
        # the workload's horizon: every member to t = to_t (a member stops at it
        # while the others go on), then the FP64 statistics of each level
        t0 = time.perf_counter()
        done = steps + warmup
        while done < 20000:
            plan.step(50, t_end=to_t)
            done += 50
            plan.synchronize()
            if min(plan.clock(m)[0] for m in range(len(Ns))) >= to_t * (1 - 1e-12):
                break
        wall = time.perf_counter() - t0
        levels = {}
        for N, M, _ in ENSEMBLE_LEVELS:
            st = plan.ensemble_stats(N, fields=False)
            levels[str(N)] = {k: st[k] for k in ("members", "energy", "energy_se", "enstrophy",
                                                 "enstrophy_se", "dissipation", "dissipation_se")}
            levels[str(N)]["steps_to_t"] = max(plan.clock(m)[1] for m in range(len(Ns)) if Ns[m] == N)
        info["to_t"] = {"t": to_t, "graph_steps": done, "wall_s_after_timed": wall, "levels": levels}
    plan.close()
    return info


# FP64 arithmetic peak of one GB300 from its unit counts: 152 SMs x 2 FP64 FMA
# (4 flops) per SM per clock x the 2070 MHz maximum SM clock = 1.259 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# FP32 pipe of one GB300: 152 SMs x 128 lanes x 2070 MHz = 40.3e12 FP32
# operations (add, mul or fma, one each) per second
FP32_OPS_PEAK_T = 152 * 128 * 2.070e9 / 1e12
# FP32 operations per FP64-equivalent flop of the FFT model in double-single
# arithmetic (ns3d_df64.cuh): a sum costs 11 (TwoSum, low parts, Dekker's
# renormalisation), a product 7 (FMA TwoProduct, cross terms, renormalisation);
# the radix codelets are two thirds sums, one third products
DF64_OPS_PER_FLOP = (2 * 11 + 7) / 3.0


def fp64_roofline(N: int, P: int, ms_per_step: float) -> dict:
    """Arithmetic roofline of an FP64 step: its long-line transforms run in
    double-single arithmetic on the FP32 pipe, so the flop model (5 P log2 P per
    line) times DF64_OPS_PER_FLOP FP32 operations is set against the FP32 pipe's
    operation rate; the FP64-equivalent rate is reported beside it."""
    flops = fft_flops_per_step(N, P)
    t = ms_per_step * 1e-3
    ach = flops * DF64_OPS_PER_FLOP / t / 1e12
    return {"bound": "alu", "pipe": "FP32 (double-single transforms)", "achieved": ach,
            "peak": FP32_OPS_PEAK_T, "peak_kind": "unit counts x max clock", "unit": "Tops/s",
            "frac": ach / FP32_OPS_PEAK_T, "flops_per_step": flops,
            "fp32_ops_per_fp64_flop": DF64_OPS_PER_FLOP,
            "fp64_equivalent_TFLOPs": flops / t / 1e12}


def fft_flops_per_step(N: int, P: int) -> float:
    """Algorithmic flops of one RK3 step: 5 P log2 P per complex line of
    length P over the line families of one right-hand side (inverse x 3 N h,
    inverse y 3 P h, z 4.5 P^2 = 1.5 inverse + 3 forward packed complex lines,
    forward y 6 P h, forward x 6 N h; h = N/2), three evaluations per step."""
    import math
    h = N // 2
    lines = 3 * N * h + 3 * P * h + 4.5 * P * P + 6 * P * h + 6 * N * h
    return 3.0 * lines * 5.0 * P * math.log2(P)


def bench_plain_fp64(B, torch, N: int, steps: int):
    """The plain FP64 path on the main workload, and the FP32 path's relative
    L2 error against it: one right-hand side, and the state after 10 steps."""
    import ns3d_inputs as I
    u0 = I.random_spectrum(N, seed=20240001)
    res = {}
    for name, dtype in (("f32", B.NS3D_F32), ("f64", B.NS3D_F64)):
        p = B.Plan([N], dtype, eps0=1.0, cfl=0.5)
        r = p.eval_rhs(0, u0).to(torch.complex128)
        p.set_initial(0, u0)
        p.step(10)
        res[name] = (r, p.get_state(0).to(torch.complex128))
        p.close()
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    err = {"rhs_rel_l2": rel(res["f32"][0], res["f64"][0]),
           "state_after_10_steps_rel_l2": rel(res["f32"][1], res["f64"][1])}
    del res
    torch.cuda.empty_cache()
    plan = B.Plan([N], B.NS3D_F64, eps0=1.0, cfl=0.5)
    plan.set_initial(0, u0)
    plan.step(1)
    plan.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    P = plan.info(0)["P"]
    plan.close()
    return {"N": N, "steps": steps, "ms_per_step": ms / steps,
            "value": N ** 3 * steps / (ms * 1e-3), "unit": UNIT, "f32_error_vs_f64": err,
            "roofline": fp64_roofline(N, P, ms / steps)}


def bench_forms(B, torch, N: int, steps: int = 5):
    """The advective (nonlinear_form = 1) and rotational (2) forms of the
    nonlinear term at N^3 FP32 (generic tile kernels; 12 and 6 inverse
    transforms instead of 3), and their relative L2 distance from the
    divergence form's state after the timed steps."""
    import ns3d_inputs as I
    u0 = I.random_spectrum(N, seed=20240001)
    out, states = {}, {}
    for name, form in (("divergence", 0), ("advective", 1), ("rotational", 2)):
        plan = B.Plan([N], B.NS3D_F32, eps0=1.0, cfl=0.5, nonlinear_form=form)
        plan.set_initial(0, u0)
        plan.step(2)
        plan.synchronize()
        plan.set_initial(0, u0)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        states[form] = plan.get_state(0).to(torch.complex128)
        plan.close()
        out[name] = {"ms_per_step": ms / steps, "value": N ** 3 * steps / (ms * 1e-3)}
        if form:
            d = torch.linalg.vector_norm(states[form] - states[0]) / torch.linalg.vector_norm(states[0])
            out[name]["state_rel_l2_vs_divergence"] = float(d)
    del states
    torch.cuda.empty_cache()
    return {"N": N, "steps": steps, "dtype": "f32", "unit": UNIT, **out}


def embedded_ic(torch, N: int, cdtype, seed: int, k0: float, n0: int = 256):
    """The random-spectrum IC (E(k) ~ k^4 exp(-2 (k/k0)^2), E = 1/2) drawn on
    an n0^3 grid and embedded into the N^3 spectrum on the device: for k0 = 8
    its energy above |k| = n0/2 is below exp(-500), so this is the N^3 field
    of that spectrum without a dense N^3 array on the host."""
    import ns3d_inputs as I
    small = torch.from_numpy(I.random_spectrum(n0, seed=seed, k0=k0)).to("cuda", cdtype)
    h0 = n0 // 2
    idx = torch.arange(n0, device="cuda")
    tgt = torch.where(idx < h0, idx, idx - n0 + N)
    big = torch.zeros((3, N, N, N // 2 + 1), dtype=cdtype, device="cuda")
    big[:, tgt[:, None], tgt[None, :], : h0 + 1] = small
    return big


def bench_largest(B, torch, cases=((1024, "f32", 4), (768, "f64", 2))):
    """The largest single-sample workloads (k0 = 8 random IC, CFL 0.5): N^3
    FP32 and FP64 on the generic kernels (P = 1536 and 1152)."""
    out = []
    for N, dt, steps in cases:
        dtype = B.NS3D_F32 if dt == "f32" else B.NS3D_F64
        cdt = torch.complex64 if dt == "f32" else torch.complex128
        rec = {"N": N, "dtype": dt, "steps": steps}
        plan = None
        try:
            plan = B.Plan([N], dtype, eps0=1.0, cfl=0.5)
            u = embedded_ic(torch, N, cdt, seed=20240005, k0=8.0)
            plan.set_initial(0, u)
            plan.synchronize()
            del u
            torch.cuda.empty_cache()
            plan.step(1)
            plan.synchronize()
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            plan.synchronize()
            kms, kn = plan.step_timed(1)
            P = plan.info(0)["P"]
            kb = kernel_bytes(N, P, 8 if dt == "f32" else 16, 1)
            step_bytes = 3 * sum(kb[k] for i, k in enumerate(KINDS) if kn[i] > 0)
            rec.update({"P": P, "ms_per_step": ms, "value": N ** 3 / (ms * 1e-3), "unit": UNIT,
                        "device_GB": plan.info(0)["device_bytes"] / 1e9,
                        "kernel_ms": {k: kms[i] / max(kn[i], 1) for i, k in enumerate(KINDS) if kn[i]},
                        "bytes_per_step_GB": step_bytes / 1e9,
                        "achieved_GBps": step_bytes / (ms * 1e-3) / 1e9})
            if dt == "f64":   # arithmetic-bound, not HBM-bound
                rec["roofline"] = fp64_roofline(N, P, ms)
        except Exception as e:   # recorded, not fatal: the main line still prints
            rec["error"] = str(e).splitlines()[0][:200]
        finally:
            if plan is not None:
                plan.close()
            torch.cuda.empty_cache()
        out.append(rec)
    return out


def cufft_pipeline(torch, N: int, L: float = 2 * math.pi, nu: float = 0.0, s: float = 1.5,
                   theta: float = 0.5, eps0: float = 1.0, dev: str = "cuda"):
    """Comparison only, not the product: the same right-hand side written with
    torch.fft (cuFFT) and element-wise torch kernels in FP32 -- zero-pad to
    P = 3N/2, c2r, the six products, r2c, truncate, -i kappa . B, Leray,
    dissipation.  Returns rhs(u) for D1-layout complex64 tensors."""
    P, h = 3 * N // 2, N // 2
    k = torch.fft.fftfreq(N, 1.0 / N, device=dev, dtype=torch.float64)
    kz = torch.arange(h + 1, device=dev, dtype=torch.float64)
    KX, KY, KZ = torch.meshgrid(k, k, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    a = 2 * math.pi / L
    kap = torch.stack([a * KX, a * KY, a * KZ]).to(torch.float32)
    kap2 = (a * a * k2)
    mN2 = float(N) ** (2 * theta)
    epsN = eps0 * float(N) ** (1 - 2 * s)
    q = torch.where(k2 > math.floor(mN2 * (1 + 1e-12)),
                    1 - (mN2 / torch.clamp(k2, min=1.0)) ** ((2 * s - 1) / (2 * theta)),
                    torch.zeros_like(k2))
    lam = (nu * kap2 + epsN * kap2 ** s * q).to(torch.float32)
    keep = ((KX.abs() < h) & (KY.abs() < h) & (KZ < h)).to(torch.float32)
    inv_k2 = torch.where(k2 > 0, 1.0 / torch.clamp(kap2, min=1e-300), torch.zeros_like(kap2)).to(torch.float32)
    rows = torch.cat([torch.arange(h, device=dev), torch.arange(P - h + 1, P, device=dev)])
    src = torch.cat([torch.arange(h, device=dev), torch.arange(N - h + 1, N, device=dev)])
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]

    def rhs(u):
        U = torch.zeros((3, P, P, P // 2 + 1), dtype=torch.complex64, device=dev)
        U[:, rows[:, None], rows[None, :], :h] = u[:, src[:, None], src[None, :], :h]
        phys = torch.fft.irfftn(U, s=(P, P, P), norm="forward")
        del U
        Bh = torch.zeros((3, 3) + u.shape[1:], dtype=torch.complex64, device=dev)
        for j, l in pairs:
            F = torch.fft.rfftn(phys[j] * phys[l], norm="forward")
            Bh[j, l, src[:, None], src[None, :], :h] = F[rows[:, None], rows[None, :], :h]
            if j != l:
                Bh[l, j] = Bh[j, l]
        b = -1j * (kap[None, 0] * Bh[:, 0] + kap[None, 1] * Bh[:, 1] + kap[None, 2] * Bh[:, 2])
        kb = (kap[0] * b[0] + kap[1] * b[1] + kap[2] * b[2]) * inv_k2
        return (b - kap * kb[None] - lam[None] * u) * keep[None]

    return rhs


def bench_cufft(torch, N: int = 256, steps: int = 5):
    """Timing of the cuFFT pipeline above, one SSP-RK3 step = three rhs calls
    (fixed dt, so no CFL reduction is timed)."""
    import ns3d_inputs as I
    rhs = cufft_pipeline(torch, N)
    u = torch.from_numpy(I.random_spectrum(N, seed=20240001)).to("cuda", torch.complex64)
    dt = 1e-3

    def step(u):
        u1 = u + dt * rhs(u)
        u2 = 0.75 * u + 0.25 * (u1 + dt * rhs(u1))
        return u / 3.0 + (2.0 / 3.0) * (u2 + dt * rhs(u2))

    u = step(u)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        u = step(u)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"kind": "comparison (torch.fft = cuFFT + element-wise torch kernels, FP32), not the product",
            "N": N, "steps": steps, "ms_per_step": ms, "value": N ** 3 / (ms * 1e-3), "unit": UNIT}


def bench_adjoint(B, torch, N: int = 128, nsteps: int = 200, every: int = 20):
    """Band-energy gradient (8 <= |k| < 16 at step `nsteps`, fixed dt) at 128^3:
    wall time of one gradient against `nsteps` forward steps, with every stage
    state kept from the forward pass (checkpoint_every = 0: 3 nsteps states in
    HBM, nothing recomputed) and with checkpoints every `every` steps (each
    segment recomputed once)."""
    import ns3d_inputs as I
    out, grads = {}, {}
    for dt_name, dtype in (("f32", B.NS3D_F32), ("f64", B.NS3D_F64)):
        plan = B.Plan([N], dtype, eps0=1.0, dt_fixed=0.005)
        plan.set_initial(0, I.random_spectrum(N, seed=20240004))
        plan.grad_band_energy(0, 8.0, 16.0, 2, checkpoint_every=2)     # warm-up
        r = {}
        for mode, C in (("kept", 0), ("checkpointed", every)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = plan.grad_band_energy(0, 8.0, 16.0, nsteps, checkpoint_every=C)
            torch.cuda.synchronize()
            r[mode] = time.perf_counter() - t0
            if mode == "kept":
                grads[dt_name] = g.to(torch.complex128)
            else:
                d = g.to(torch.complex128) - grads[dt_name]
                r["modes_rel_l2"] = float(torch.linalg.vector_norm(d) /
                                          torch.linalg.vector_norm(grads[dt_name]))
            del g
        plan.step(2)
        plan.synchronize()
        t0 = time.perf_counter()
        plan.step(nsteps)
        plan.synchronize()
        tf = time.perf_counter() - t0
        plan.close()
        out[dt_name] = {"gradient_s": r["kept"], "forward_s": tf, "ratio": r["kept"] / tf,
                        "checkpointed_gradient_s": r["checkpointed"],
                        "checkpointed_ratio": r["checkpointed"] / tf,
                        "kept_vs_checkpointed_rel_l2": r["modes_rel_l2"]}
    d = grads["f32"] - grads["f64"]
    out["f32_gradient_rel_l2_vs_f64"] = float(torch.linalg.vector_norm(d) /
                                              torch.linalg.vector_norm(grads["f64"]))
    return {"N": N, "steps": nsteps, "checkpoint_every": {"kept": 0, "checkpointed": every},
            "kept_states_GB": {"f32": 3 * nsteps * 3 * N * N * (N // 2) * 8 / 1e9,
                               "f64": 3 * nsteps * 3 * N * N * (N // 2) * 16 / 1e9}, **out}


def bench_mesh_refinement(B, torch, levels=(64, 128), ref_N: int = 256, members: int = 16,
                          t_end: float = 1.0):
    """Mesh refinement of section 6.1: the perturbed Taylor-Green initial
    measure on the unit torus (s = 1.5, nu = 0), `members` samples at each
    coarse resolution and at the reference resolution ref_N, all in one FP32
    plan run to t_end with per-member CFL steps; then, per coarse level, the
    1-point Wasserstein distance, mean, variance and paired sample errors
    against the reference on the coarse grid points, with the Monte Carlo
    error bar of the mean difference (ns3d_mesh_refinement)."""
    Ns = [N for N in tuple(levels) + (ref_N,) for _ in range(members)]
    # on the unit torus kappa = 2 pi k: eps0 = (2 pi)^(-2s) gives each mode the
    # damping eps_N |k|^(2s) of the 2 pi-periodic workloads (lambda_max dt ~ 0.3
    # at CFL 0.5, where eps0 = 1 would exceed the RK3 limit)
    eps0 = (2 * math.pi) ** -3.0
    plan = B.Plan(Ns, B.NS3D_F32, L=1.0, eps0=eps0, cfl=0.5)
    try:
        return _mesh_refinement_run(plan, Ns, levels, ref_N, members, t_end)
    finally:
        plan.close()
        torch.cuda.empty_cache()


def _mesh_refinement_run(plan, Ns, levels, ref_N, members, t_end):
    import ns3d_inputs as I
    for i, N in enumerate(Ns):
        plan.set_initial(i, I.perturbed_taylor_green(N, seed=20240061, member=i % members))
        plan.project(i)                   # the flow starts from the divergence-free part
    t0 = time.perf_counter()
    steps = 0
    while steps < 20000:
        plan.step(50, t_end=t_end)
        steps += 50
        plan.synchronize()
        if min(plan.clock(m)[0] for m in range(len(Ns))) >= t_end * (1 - 1e-12):
            break
    wall = time.perf_counter() - t0
    out = {"initial_measure": "perturbed Taylor-Green (section 6.1), L = 1, eps0 = (2 pi)^-3",
           "members": members,
           "reference_N": ref_N, "t": t_end, "graph_steps": steps, "wall_s": wall, "dtype": "f32",
           "levels": {}}
    for N in levels:
        r = plan.mesh_refinement(N, ref_N)
        out["levels"][str(N)] = {k: r[k] for k in ("w1", "mean_err", "var_err", "sample_err", "mc_se")}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--members", type=int, default=1, help="members per GPU at N")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-ensemble and FP64 comparison lines")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- byte model

def kernel_bytes(N: int, P: int, esz: int, members: int):
    """Algorithmic bytes per launch of each kernel kind (compulsory reads and
    writes of its input and output arrays; complex elements of esz bytes)."""
    h = N // 2
    U = 3 * N * N * h
    A = 3 * P * N * h
    Bq = 3 * P * h * P
    Cq = 6 * P * h * P
    Dq = 6 * P * N * h
    Bh = 6 * N * N * h
    per = {
        "inverse_x": U + A,
        "inverse_y": A + Bq,
        "zpass": Bq + Cq,
        "forward_y": Cq + Dq,
        "forward_x": Dq + Bh,
        "spectral": Bh + U + U + (2 * U) / 3.0,   # stages 2, 3 also read the stage state
        # forward x + spectral step + RK3 combine + next stage's inverse x
        "fused_x": Dq + U + U + (2 * U) / 3.0 + A,
    }
    return {k: v * esz * members for k, v in per.items()}


KINDS = ["inverse_x", "inverse_y", "zpass", "forward_y", "forward_x", "spectral"]

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from one ncu
# capture of the same command on GB300, keyed (kind, N, dtype, members), with the profiles/
# file that records the capture; an entry is removed when its kernel changes after the capture
NCU_TRAFFIC = {("zpass", 256, "f32", 1): (453.16e6 + 845.25e6, "profiles/zpass_256cube_f32.md")}


def window_sizes(steps: int, n: int = 5, min_steps: int = 20):
    """The timed steps split into n consecutive windows of at least min_steps
    each (one window when there are too few steps); the sizes sum to steps."""
    n = max(1, min(n, steps // min_steps))
    return [steps // n + (1 if i < steps % n else 0) for i in range(n)]


def traffic_entry(kind: str, N: int, dtype: str, members: int):
    """(bytes, source) of the ncu capture for this kernel and workload, or (None, None)."""
    return NCU_TRAFFIC.get((kind, N, dtype, members), (None, None))


# ----------------------------------------------------------------------------- oracle timing

_ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_member_step(args):
    """Seconds of one oracle RK3 step of member `member` of the N^3 random
    workload (runs in a pool worker; one thread each)."""
    N, member = args
    import ns3d_inputs as I
    from oracle import solver as S
    u = I.random_spectrum(N, seed=20240001, member=member)
    prm = S.Params(eps0=1.0, cfl=0.5)
    t = time.perf_counter()
    S.rk3_step(u, prm)
    return time.perf_counter() - t


def oracle_sample_seconds(N: int, steps: int = 1, taylor_green: bool = False) -> float:
    """Wall seconds of `steps` oracle RK3 steps at N^3 in a fresh single-threaded
    process: the random-spectrum sample (CFL 0.5), or the Taylor-Green vortex
    with nu = 0.01 and dt = 0.01 (the 32^3 FP64 case)."""
    if taylor_green:
        setup = ("u = I.taylor_green(%d)\n"
                 "prm = S.Params(nu=0.01, eps0=1.0, dt_fixed=0.01)\n" % N)
    else:
        setup = ("u = I.random_spectrum(%d, seed=20240001)\n"
                 "prm = S.Params(eps0=1.0, cfl=0.5)\n" % N)
    code = (
        "import time, sys; sys.path.insert(0, %r)\n"
        "import ns3d_inputs as I\n"
        "from oracle import solver as S\n" % ROOT + setup +
        "S.rk3_step(u, prm)\n"
        "t = time.perf_counter()\n"
        "S.integrate(u, prm, %d)\n"
        "print(time.perf_counter() - t)\n" % steps)
    env = dict(os.environ, **_ONE_THREAD)
    out = subprocess.run([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, text=True,
                         check=True)
    return float(out.stdout.strip().splitlines()[-1])


def oracle_all_cores(N: int, workers: int):
    """Ensemble throughput of the oracle on all host cores: `workers`
    single-threaded spawn-started processes, each advancing its own member by
    one RK3 step (members are independent, Algorithm 1), timed from the first
    submission to the last result after a warm-up round."""
    import concurrent.futures as cf
    import multiprocessing as mp
    old = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update(_ONE_THREAD)            # inherited by the spawned workers
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_member_step, [(16, m) for m in range(workers)]))   # imports, warm-up
            t = time.perf_counter()
            list(ex.map(_oracle_member_step, [(N, m) for m in range(workers)]))
            return time.perf_counter() - t
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def host_cpu():
    """CPU model and logical core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, text=True).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


def cpu_baseline():
    """The FP64 numpy oracle on this host's cores (a reported baseline, not a
    target): the random-spectrum workload one RK3 step at 64^3 single-threaded
    and as an ensemble on all cores, and 20 of the 32^3 Taylor-Green case's
    100 steps single-threaded."""
    N = 64
    model, ncpu = host_cpu()
    sec1 = oracle_sample_seconds(N, 1)
    workers = max(1, ncpu)
    secw = oracle_all_cores(N, workers)
    tg_steps = 20
    sec_tg = oracle_sample_seconds(32, tg_steps, taylor_green=True)
    return {"value": workers * N ** 3 / secw, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} members of the random-spectrum workload at {N}^3 (P = 96), one "
                      f"SSP-RK3 step each, one single-threaded process per core, all at once: "
                      f"{secw:.2f} s wall",
            "cpu_model": model, "nproc": ncpu,
            "single_thread": {"value": N ** 3 / sec1, "unit": UNIT, "cores": 1,
                              "sample": f"one SSP-RK3 step at {N}^3, one thread: {sec1:.2f} s"},
            "taylor_green_32": {"value": 32 ** 3 * tg_steps / sec_tg, "unit": UNIT, "cores": 1,
                                "sample": f"{tg_steps} of the 100 fixed steps (dt = 0.01, nu = 0.01) "
                                          f"of the 32^3 FP64 Taylor-Green case, one thread: "
                                          f"{sec_tg:.2f} s"},
            "not_run": "256^3 (one oracle right-hand side takes minutes on one core): the 64^3 "
                       "sample of the same initial-data family stands for it, per grid point"}


def oracle_step_seconds(N: int, warmup: int, steps: int):
    """Per-step wall seconds of `steps` oracle RK3 steps at N^3 after `warmup`
    untimed ones, all in one fresh single-threaded process."""
    code = (
        "import time, sys; sys.path.insert(0, %r)\n"
        "import ns3d_inputs as I\n"
        "from oracle import solver as S\n"
        "u = I.random_spectrum(%d, seed=20240001)\n"
        "prm = S.Params(eps0=1.0, cfl=0.5)\n"
        "for _ in range(%d): u = S.rk3_step(u, prm)[0]\n"
        "for _ in range(%d):\n"
        "    t = time.perf_counter(); u = S.rk3_step(u, prm)[0]; print(time.perf_counter() - t)\n"
        % (ROOT, N, warmup, steps))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, text=True,
                         check=True)
    return [float(x) for x in out.stdout.split()]


def run_reference(args, rank, world):
    if rank != 0:
        return
    N = 16      # one oracle RK3 step at 16^3 per timed step: the whole run stays within minutes
    per = oracle_step_seconds(N, args.warmup, args.steps)
    tot = sum(per)
    value = N ** 3 * args.steps / tot
    model, ncpu = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{N}^3 random-spectrum sample (k0 = 4, E = 0.5), CFL 0.5, "
                               "hyper-viscosity s = 1.5, theta = 1/2: a bounded sample of the "
                               f"{args.N}^3 workload, same initial-data family and parameters, "
                               "compared per grid point",
                   "N": N, "sample_of_N": args.N, "members_per_gpu": 1, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cpu_model": model, "nproc": ncpu,
                         "sample": f"each step is one SSP-RK3 step of the FP64 numpy oracle at {N}^3 "
                                   "(the paper publishes no code to run), single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import ns3d_inputs as I
    from paper_2401_09843_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    N, M = args.N, args.members
    dtype = B.NS3D_F32 if args.dtype == "f32" else B.NS3D_F64
    esz = 8 if dtype == B.NS3D_F32 else 16
    stream = torch.cuda.current_stream()
    plan = B.Plan([N] * M, dtype, eps0=1.0, cfl=0.5)
    P = plan.info(0)["P"]
    if N <= 256:
        u0 = [I.random_spectrum(N, seed=20240001 + rank * 1000 + m) for m in range(M)]
    else:   # the largest workload: k0 = 8 spectrum, built on the device
        cdt = torch.complex64 if dtype == B.NS3D_F32 else torch.complex128
        u0 = [embedded_ic(torch, N, cdt, seed=20240005 + rank * 1000 + m, k0=8.0) for m in range(M)]
        args.no_e2e = True
    for m in range(M):
        plan.set_initial(m, u0[m])

    # warm-up (graph capture happens here)
    plan.step(args.warmup)
    plan.synchronize()

    smi_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    clocks = ClockSampler(smi_index)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    time.sleep(0.25)
    # the K steps in consecutive windows, an event between windows (ns3d_step
    # only enqueues graph replays, so the windows run back to back)
    wins = window_sizes(args.steps)
    wev = [torch.cuda.Event(enable_timing=True) for _ in range(len(wins) - 1)]
    e0.record(stream)
    for i, k in enumerate(wins):
        plan.step(k)
        (wev[i] if i < len(wev) else e1).record(stream)
    torch.cuda.synchronize()
    time.sleep(0.1)
    ck = clocks.stop()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    bounds = [e0] + wev + [e1]
    win_ms = [bounds[i].elapsed_time(bounds[i + 1]) / k for i, k in enumerate(wins)]
    status_ok = True
    try:
        plan.synchronize()
    except B.Ns3dError:
        status_ok = False
    launches = plan.info(0)["launches_per_step"] * args.steps

    # per-kernel durations: same kernels, eager, CUDA events on the plan's stream
    kms, kn = plan.step_timed(max(3, min(20, args.steps // 10)))
    kb = kernel_bytes(N, P, esz, M)
    # a level with the fused x pass reports no inverse-x / forward-x launches
    # and its fused kernel under the spectral slot
    fused = kn[0] == 0 and kn[4] == 0 and kn[5] > 0
    kinds = list(KINDS)
    if fused:
        kinds[5] = "fused_x"
    per_kind = {}
    for i, k in enumerate(kinds):
        if kn[i] == 0:
            continue
        avg = kms[i] / kn[i]
        per_kind[k] = {"ms": avg, "GBps": kb[k] / (avg * 1e-3) / 1e9 if avg > 0 else None}
    dom = max(range(6), key=lambda i: kms[i])
    peak, peak_kind = measured_peaks()
    dom_ms = kms[dom] / max(kn[dom], 1)
    ach = kb[kinds[dom]] / (dom_ms * 1e-3) / 1e9
    step_bytes = 3 * sum(kb[k] for i, k in enumerate(kinds) if kn[i] > 0)
    step_ms_eager = sum(kms) / max(kn[5] / 3, 1)

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        npd = np.complex64 if dtype == B.NS3D_F32 else np.complex128
        hin = [torch.from_numpy(np.ascontiguousarray(u.astype(npd))).pin_memory().numpy() for u in u0]
        hout = [torch.empty(u.shape, dtype=plan.cdtype).pin_memory().numpy() for u in u0]
        nb = sum(h.nbytes for h in hin)
        ke = max(3, min(20, args.steps // 10))
        # serial: copy in, one step, copy out, one after another on the plan's stream
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            for m in range(M):
                plan.set_initial_host(m, hin[m])
            plan.step(1)
            for m in range(M):
                plan.get_state_host(m, hout[m])
        t1 = time.perf_counter()
        et_serial = max_over_ranks(t1 - t0)
        # pipelined: a second plan on its own stream; the two alternate, so one
        # plan's host copies run while the other's step computes.  Every step
        # still uploads its input and downloads its result.
        plan2 = B.Plan([N] * M, dtype, eps0=1.0, cfl=0.5, stream=torch.cuda.Stream())
        for m in range(M):
            plan2.set_initial_host(m, hin[m])
        plan2.step(1)                      # captures plan2's graph
        plan2.synchronize()
        plans = (plan, plan2)
        outs = (hout, [torch.empty(u.shape, dtype=plan.cdtype).pin_memory().numpy() for u in u0])
        serial_out = [h.copy() for h in hout]
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for m in range(M):
            plans[0].set_initial_host(m, hin[m])
        plans[0].step(1)
        for k in range(1, ke):
            X, Y = plans[k % 2], plans[(k - 1) % 2]
            for m in range(M):
                X.set_initial_host(m, hin[m])
            X.step(1)
            for m in range(M):
                Y.get_state_host(m, outs[(k - 1) % 2][m])
        for m in range(M):
            plans[(ke - 1) % 2].get_state_host(m, outs[(ke - 1) % 2][m])
        t1 = time.perf_counter()
        et = max_over_ranks(t1 - t0)
        same = all(np.array_equal(o[m], serial_out[m]) for o in outs for m in range(M))
        plan2.close()
        e2e = {"value": world * M * N ** 3 * ke / et, "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "pipeline": "two plans on two streams alternate: one sample's host copies "
                           "overlap the other's step",
               "results_equal_serial": same,
               "serial_value": world * M * N ** 3 * ke / et_serial}

    value = world * M * N ** 3 * args.steps / (ms * 1e-3)
    if rank != 0:
        plan.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": f"{N}^3 random-spectrum sample{'s' if M > 1 else ''} per GPU "
                               f"(k0 = {4 if N <= 256 else 8}, E = 0.5), CFL 0.5, hyper-viscosity s = 1.5, "
                               f"theta = 1/2",
                   "N": N, "P": P, "members_per_gpu": M,
                   "l2": "no flush: each step streams ~%.1f GB through HBM (> 126 MB L2)" % (step_bytes / 1e9),
                   "parallelism": f"{world} GPU(s), one sample each (ensemble shards)"},
        "samples_steps_per_s": world * M * args.steps / (ms * 1e-3),
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": kinds[dom], "achieved": ach, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                     "bytes_per_launch": kb[kinds[dom]],
                     "traffic": traffic_entry(kinds[dom], N, args.dtype, M)[0],
                     "traffic_source": traffic_entry(kinds[dom], N, args.dtype, M)[1]},
        "windows": {"steps": wins, "ms_per_step": win_ms,
                    "median_ms_per_step": float(statistics.median(win_ms))},
        "step_roofline": {"bytes_per_step": step_bytes,
                          "achieved_GBps": step_bytes / (ms / args.steps * 1e-3) / 1e9,
                          "frac": step_bytes / (ms / args.steps * 1e-3) / 1e9 / peak},
        "kernels": per_kind,
        "eager_ms_per_step": step_ms_eager,
        "clocks": ck,
        "e2e": e2e,
        "status_ok": status_ok,
    }
    if not args.no_extras and world == 1:
        extras = [("batched_ensemble", lambda: bench_ensemble(B, torch, steps=10, warmup=2, to_t=1.0)),
                  ("plain_fp64", lambda: bench_plain_fp64(B, torch, N, steps=3)),
                  ("nonlinear_forms", lambda: bench_forms(B, torch, N)),
                  ("largest", lambda: bench_largest(B, torch)),
                  ("cufft_pipeline", lambda: bench_cufft(torch, N)),
                  ("adjoint", lambda: bench_adjoint(B, torch)),
                  ("mesh_refinement", lambda: bench_mesh_refinement(B, torch))]
        for name, run in extras:
            try:        # an extra line that fails is recorded; the main line still prints
                line[name] = run()
            except Exception as e:
                line[name] = {"error": str(e).splitlines()[0][:200]}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
