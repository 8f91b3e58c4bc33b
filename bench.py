"""Benchmark: CSS density-matrix P build time per geometry, 10,000 water-like molecules.

Workload (synthetic, seeded): 10,000 molecules in a 66.9 A periodic box, 23 orbitals per
molecule (N = 230,000), 6 A coupling cut-off, colouring radius R_col = 10 A, block-Lanczos
depth m = 40, Fermi-Dirac kT = 0.05 eV, mu from the Ritz quadrature of Tr P = N_e/2; an
MD-like sequence of 20 geometries (Gaussian steps of 0.02 A) with H rebuilt per geometry.
One step = one P build = css_color + css_probes + css_density on the next geometry, with H
and the positions already resident in HBM (H: 1.17 GB in FP64, larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl ours|reference]

Multi-GPU (torchrun): every rank builds P for its own geometries (independent problems, no
data-path collective); the time is the maximum over ranks and `value` is that time divided
by the P builds of all ranks.  `--impl reference` times the CPU oracle on a bounded sample
(one colour of the P build, both Lanczos passes, scaled to all colours) on rank 0 only.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "P build s/step at 10k H2O"
SPMM_KERNEL_VERSION = "k_spmm_dup-v2"  # profiles/spmm_traffic.json must name the kernel measured


def hv_kernel(mixed, b, tc=False):
    """(name, version tag) of the H*V kernel a build runs: the tensor-core one when asked for, the
    exact-width FP32 kernel for b = 6 and 23, else the padded FFMA/DFMA kernel."""
    if mixed and (tc or os.environ.get("CSS_HV_TC") == "1") and 16 < b <= 24:
        return "k_hv_tc (H*V on tcgen05, 3xTF32)", "k_hv_tc"
    if mixed and b in (6, 23) and not os.environ.get("CSS_SPMM_VARIANT"):
        return ("k_spmm_dup (exact-width H*V on the FP32 FMA pipe, packed row pairs, all colours of the "
                "system as columns)", SPMM_KERNEL_VERSION)
    return ("k_spmm (padded H*V on the " + ("FP32 FMA" if mixed else "FP64 DFMA") +
            " pipe, all colours of the system as columns)", "k_spmm-padded")
FP64_PEAK_NOTE = "FP64 peak: 1.25 TFLOP/s nominal GB300 FP64 rate"
FP64_PEAK = 1.25                                 # TFLOP/s


def measured_peaks():
    """HBM GB/s, dense BF16 TF/s (burst, sustained) and the maximum SM clock from
    MEASURED_PEAKS.json, else the fallback figures of an earlier GB300 measurement."""
    p = ROOT / "MEASURED_PEAKS.json"
    try:
        d = json.loads(p.read_text())
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "sm_max_mhz": 2070.0,
                "source": "of fallback"}


def fp32_peak_tflops(n_sm: int, sm_max_mhz: float) -> float:
    """FFMA peak: SMs x 128 FP32 lanes x 2 flop x maximum SM clock."""
    return n_sm * 128 * 2 * sm_max_mhz * 1e6 / 1e12


def tf32_peak_tflops(pk) -> float:
    """Dense TF32 tensor peak: the measured sustained BF16 rate x the nominal TF32 / BF16 ratio
    (1.1 / 2.25 PFLOP/s dense)."""
    return pk["bf16_sustained"] * 1.1 / 2.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64", "3xtf32", "fp64-split"], default="mixed")
    ap.add_argument("--n-mol", type=int, default=10000)
    ap.add_argument("--kind", default="dzp")
    ap.add_argument("--m", type=int, default=40)
    ap.add_argument("--r-col", type=float, default=10.0)
    ap.add_argument("--geometries", type=int, default=20)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the energy-weighted and S^-1/2 timings")
    ap.add_argument("--oracle-full", action="store_true",
                    help="reference arm: time complete oracle builds instead of the scaled sample")
    ap.add_argument("--workload", choices=["md10k", "million"], default="md10k",
                    help="million: the 10^6-molecule, 6-orbital streamed two-pass build (its own JSON line)")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"CSS P build, {a.n_mol} water-like molecules, {23 if a.kind == 'dzp' else 6} orbitals "
                        f"each, MD-like sequence of {a.geometries} geometries",
            "n_mol": a.n_mol, "orbitals_per_molecule": 23 if a.kind == "dzp" else 6, "krylov_blocks_m": a.m,
            "r_col_A": a.r_col, "coupling_cutoff_A": 6.0, "kT_eV": 0.05, "geometries": a.geometries,
            "precision": a.precision}


def l2_note(H):
    gb = H.nnzb * H.b * H.b * 8 / 1e9
    return (f"inputs larger than L2: H alone is {gb:.2f} GB in FP64 and every Krylov block "
            f"{H.n_brow * H.b * H.b * 4 / 1e6:.0f} MB per colour in FP32 (the Lanczos step streams three "
            f"such blocks for every colour of the system), against a 129 MB L2")


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def build_inputs(a, indices):
    """Geometries of the MD-like sequence at `indices` (mod a.geometries) and their H."""
    from paper_2605_20918_gb300 import synth
    want = sorted({i % a.geometries for i in indices})
    geoms, cache = {}, {}
    for t, g in enumerate(synth.md_sequence(a.n_mol, max(want) + 1)):
        if t in want:
            geoms[t] = (g, synth.hamiltonian(g, a.kind, cache=cache))
    return geoms


def colour_reuse(ctx, xyz_seq, box, r_col, colour, skins=(0.0, 0.25), seed=1004):
    """Colouring kept across consecutive MD geometries with css_color_update (a blocking call):
    per skin, how many geometries had to be recoloured, the final colour count, and the mean
    host time of an update that kept the colouring (one conflict check) and of one that
    recoloured (check + colouring at R_col + skin)."""
    out = {}
    for skin in skins:
        nc, keep_ms, recolour_ms = 0, [], []
        for xyz in xyz_seq:
            t0 = time.perf_counter()
            nc, re = ctx.color_update(xyz, box, r_col, seed, colour, nc, skin=skin)
            (recolour_ms if re else keep_ms).append(1e3 * (time.perf_counter() - t0))
        out[f"skin_{skin:g}_A"] = {
            "geometries": len(xyz_seq), "recoloured": len(recolour_ms), "n_colours": int(nc),
            "ms_keep": statistics.mean(keep_ms) if keep_ms else None,
            "ms_recolour": statistics.mean(recolour_ms[1:]) if len(recolour_ms) > 1 else None}
    return out


SAMPLE_M = 2  # block-Lanczos steps per pass in the oracle sample


def oracle_sample(H, col, sign, nc, a):
    """A bounded sample of one oracle P build on the host cores, scaled to the whole build.

    The oracle runs colours in parallel (OpenMP, one thread per colour, each colour's two
    block-Lanczos passes and two exact diagonalisations of its m b x m b projected matrix on one
    thread).  The sample runs the same schedule on its first `threads` colours with depth
    SAMPLE_M instead of m (a fixed mu, so no colour waits for the others), and times one exact
    diagonalisation of an m b x m b symmetric matrix; the build is then
        t_lanczos x (m / SAMPLE_M) x ceil(nc / threads) + 2 x ceil(nc / threads) x t_eig.
    mu, the extraction and the symmetrisation (a few percent of a build) are not in it."""
    import oracle
    threads = oracle.num_threads()
    flags = oracle.REORTH_LOCAL if a.precision in ("mixed", "3xtf32") else 0
    sub = list(range(min(threads, nc)))
    t0 = time.perf_counter()
    oracle.density(H, col, sign, nc, mu=-4.0, kT=0.05, solve_mu=False, m=SAMPLE_M, flags=flags, colour_subset=sub)
    t_l = time.perf_counter() - t0
    n = a.m * H.b
    rng = np.random.default_rng(7)
    A = rng.standard_normal((n, n))
    t0 = time.perf_counter()
    oracle.eigh(A + A.T)
    t_e = time.perf_counter() - t0
    rounds = -(-nc // threads)
    est = t_l * (a.m / SAMPLE_M) * rounds + 2 * rounds * t_e
    return est, {"t_lanczos_s": t_l, "t_eig_s": t_e, "threads": threads, "colours": nc, "rounds": rounds}


def sample_note(a, parts):
    reo = ", local reorthogonalisation" if a.precision in ("mixed", "3xtf32") else ""
    return (f"oracle (FP64{reo}) on geometry 0 of the {a.n_mol}-molecule workload, its own schedule (OpenMP over "
            f"colours, one thread per colour): {parts['threads']} colours at Krylov depth {SAMPLE_M} "
            f"({parts['t_lanczos_s']:.2f} s) and one exact diagonalisation of a {a.m * 23 if a.kind == 'dzp' else a.m * 6}"
            f"-square projected matrix ({parts['t_eig_s']:.2f} s), scaled to depth {a.m} and {parts['colours']} "
            f"colours ({parts['rounds']} rounds of {parts['threads']} threads, two passes); mu and the extraction "
            f"are not in the sample")


def oracle_full_build(H, col, sign, nc, a):
    """Wall time of one complete oracle P build (mu solved), for checking the sample's scaling."""
    import oracle
    from paper_2605_20918_gb300 import synth
    flags = oracle.SYMMETRIZE | (oracle.REORTH_LOCAL if a.precision in ("mixed", "3xtf32") else 0)
    t0 = time.perf_counter()
    oracle.density(H, col, sign, nc, kT=0.05, n_elec=synth.n_electrons(H.n_brow), m=a.m, flags=flags)
    return time.perf_counter() - t0


def mode_4096(a, ctx, css, synth, dev, stream):
    """The 4,096-molecule, 23-orbital workload (N = 94,208, R_col = 10 A, m = 40): FP64 and mixed P
    builds side by side, each timed with CUDA events, with errors against the oracle's stored
    unsymmetrised columns of two colours at mu = -4 eV (tests/golden/make_fullsize_golden.py
    --n-mol 4096) and mixed against FP64 with mu solved in each."""
    import torch
    gold = ROOT / "tests" / "golden" / "fullsize_4096_colours.npz"
    g = synth.water_box(4096)
    H = synth.hamiltonian(g, "dzp")
    Hd = css.DeviceBSR.from_host(H, dev)
    xyz = torch.as_tensor(g.pos, device=dev)
    col = torch.empty(4096, dtype=torch.int32, device=dev)
    sign = torch.empty(4096 * H.b, dtype=torch.int8, device=dev)
    ne = synth.n_electrons(4096)
    out, P = {}, {}
    for pname, p in (("fp64", css.CSS_FP64), ("mixed", css.CSS_MIXED_FP32)):
        P[pname] = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev)
        nc = ctx.color(xyz, g.box, a.r_col, 1004, col)
        ctx.probes(col, H.b, 1005, sign)
        ctx.density(Hd, col, sign, nc, P[pname], kT=0.05, n_elec=ne, m=a.m, precision=p)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 1 if p == css.CSS_FP64 else 3
        e0.record(stream)
        for _ in range(reps):
            nc = ctx.color(xyz, g.box, a.r_col, 1004, col)
            ctx.probes(col, H.b, 1005, sign)
            r = ctx.density(Hd, col, sign, nc, P[pname], kT=0.05, n_elec=ne, m=a.m, precision=p)
        e1.record(stream)
        torch.cuda.synchronize()
        out[pname] = {"s_per_pbuild": e0.elapsed_time(e1) / 1e3 / reps, "mu": r["mu"], "trP": r["trP"],
                      "dTrP_vs_ne2": r["trP"] - ne / 2, "n_colours": nc, "trPH": r["trPH"]}
    out["mixed_vs_fp64_mu_solved"] = {
        "max_abs_dP": float((P["mixed"] - P["fp64"]).abs().max().item()),
        "dE_band_eV_per_molecule": abs(2 * (out["mixed"]["trPH"] - out["fp64"]["trPH"])) / 4096,
        "dmu_eV": out["mixed"]["mu"] - out["fp64"]["mu"]}
    if gold.exists():
        gd = np.load(gold)
        ch = col.cpu().numpy()
        rows = np.repeat(np.arange(H.n_brow), np.diff(H.row_ptr))
        for pname, p in (("fp64", css.CSS_FP64), ("mixed", css.CSS_MIXED_FP32)):
            ctx.density(Hd, col, sign, nc, P[pname], mu=float(gd["mu"]), kT=0.05, solve_mu=False, m=a.m,
                        precision=p, flags=0)
            Ph = None
            e = {}
            for c in gd["colours"]:
                c = int(c)
                got = P[pname][torch.as_tensor(gd[f"blocks_{c}"], device=dev)].cpu().numpy()
                if Ph is None:
                    Ph = P[pname].cpu().numpy()
                mask = ch[H.col_idx] == c
                diag = mask & (rows == H.col_idx)
                e[f"colour_{c}"] = {
                    "max_abs_dP_sampled": float(np.abs(got - gd[f"P_{c}"]).max()),
                    "dTrP_colour": float(np.trace(Ph[diag], axis1=1, axis2=2).sum()) - float(gd[f"trP_{c}"]),
                    "dE_band_colour_eV_per_molecule": abs(2 * (float((Ph[mask] * H.val[mask]).sum()) -
                                                             float(gd[f"trPH_{c}"]))) / 4096}
            out[pname]["vs_oracle_fixed_mu"] = e
        out["oracle_note"] = ("oracle's unsymmetrised columns of the first and last colour at mu = -4 eV: 32 sampled "
                              "blocks each, and the colour's share of Tr P and Tr(PH) over all its blocks")
    del P, Hd
    return out


def row_roofline(a, H, nc, rows_ms, fp32, pk):
    """Row work of one Lanczos step (everything between two H*V launches) against HBM: the
    algorithmic minimum is reading Q_{j-1}, Q_j and W = H Q_j and writing Q_{j+1} once (four
    N x w passes); the FP32 row passes of b <= 24 stream eleven (the CholeskyQR3 Grams re-read W1)."""
    w = nc * H.b
    s = 4 if fp32 else 8
    alg = 4.0 * H.n_brow * H.b * w * s
    achieved = alg / (rows_ms * 1e-3) / 1e9 if rows_ms > 0 else None
    return {"kernel": "Lanczos row work per step (three-term update, reorthogonalisation, CholeskyQR3, sampled rows)",
            "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"] if achieved else None, "ms_per_step": rows_ms,
            "alg_bytes_per_step": alg, "streamed_bytes_per_step": (11 if fp32 and 16 < H.b <= 24 else 14) / 4 * alg,
            "peak_source": f"HBM copy bandwidth {pk['source']}"}


def run_reference(a):
    """Oracle on host cores; each step one bounded sample of the P build, scaled to a whole build
    (with --oracle-full: one complete oracle build per step)."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    geoms = build_inputs(a, [0])
    g, H = geoms[0]
    col, nc = oracle.color(g.pos, g.box, a.r_col, 1004)
    sign = oracle.probes(col, H.b, 1005)
    threads = oracle.num_threads()
    times, parts = [], None
    for i in range(a.warmup + a.steps):
        if a.oracle_full:
            t = oracle_full_build(H, col, sign, nc, a)
        else:
            t, parts = oracle_sample(H, col, sign, nc, a)
        if i >= a.warmup:
            times.append(t)
    value = statistics.mean(times)
    cfg = workload_config(a)
    cfg["l2"] = l2_note(H)
    cfg["precision"] = "fp64 (CPU oracle" + (", local reorthogonalisation as the mixed GPU path)" if a.precision in ("mixed", "3xtf32")
                                             else ")")
    note = (f"one complete oracle P build of the {a.n_mol}-molecule workload per step" if a.oracle_full
            else sample_note(a, parts))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/P-build",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "s/P-build", "cores": threads, "kind": "oracle",
                             "sample": note},
            "e2e": {"value": value, "unit": "s/P-build", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(a, g, H):
    """The reference arm's sample (the same colours, depth and scaling), on geometry 0."""
    import oracle
    oracle.build()
    col, nc = oracle.color(g.pos, g.box, a.r_col, 1004)
    sign = oracle.probes(col, H.b, 1005)
    est, parts = oracle_sample(H, col, sign, nc, a)
    return {"value": est, "unit": "s/P-build", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": sample_note(a, parts)}


def run_million(a):
    """The 10^6-molecule workload (6 orbitals, N = 6,000,000, box ~310 A, R_col = 10 A, m = 30):
    mixed precision with the regenerating second block-Lanczos pass (no sampled rows stored),
    timed with CUDA events over the whole P build (colour + probes + density); the band energy
    per molecule and Tr P per molecule are compared with the oracle's on a 512-molecule system from
    the same generator (tests/golden/make_subsample_golden.py)."""
    os.environ.setdefault("CSS_TIMING", "1")
    import torch
    import paper_2605_20918_gb300 as css
    from paper_2605_20918_gb300 import build as cbuild
    from paper_2605_20918_gb300 import synth
    cbuild.build()
    n = 1_000_000
    t0 = time.perf_counter()
    g = synth.water_box(n)
    H = synth.hamiltonian(g, "minimal")
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    Hd = css.DeviceBSR.from_host(H, dev)
    xyz = torch.as_tensor(g.pos, device=dev)
    colour = torch.empty(n, dtype=torch.int32, device=dev)
    sign = torch.empty(n * H.b, dtype=torch.int8, device=dev)
    P = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev)
    ne = synth.n_electrons(n)
    ctx = css.Context(0)
    stream = torch.cuda.current_stream(dev)
    flags = css.CSS_SYMMETRIZE | css.CSS_TWO_PASS

    def step():
        nc = ctx.color(xyz, g.box, 10.0, 1004, colour)
        ctx.probes(colour, H.b, 1005, sign)
        return ctx.density(Hd, colour, sign, nc, P, kT=0.05, n_elec=ne, m=30, precision=css.CSS_MIXED_FP32,
                           flags=flags), nc

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            r, nc = step()
        e1.record(stream)
        torch.cuda.synchronize()
    value = e0.elapsed_time(e1) / 1e3 / a.steps
    inf = ctx.info()
    pk = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    achieved = inf["spmm_flops"] / (inf["ms_spmm"] * 1e-3) / 1e12 if inf["ms_spmm"] > 0 else None
    line = {"metric": "P build s/step at 10^6 H2O (6 orbitals, streamed two-pass)", "value": value,
            "unit": "s/P-build", "n_gpus": 1, "steps": a.steps, "warmup": max(a.warmup, 1), "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "CSS P build, 1,000,000 water-like molecules, 6 orbitals each (N = 6,000,000), "
                                   "two-pass block-Lanczos", "n_mol": n, "orbitals_per_molecule": 6,
                       "krylov_blocks_m": 30, "r_col_A": 10.0, "coupling_cutoff_A": 6.0, "kT_eV": 0.05,
                       "precision": "mixed", "l2": l2_note(H)},
            "roofline": {"kernel": hv_kernel(True, 6)[0], "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak_tflops(n_sm, pk["sm_max_mhz"]), "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak_tflops(n_sm, pk["sm_max_mhz"]) if achieved else None,
                         "launch_ms": inf["ms_spmm"], "launches_per_build": inf["spmm_launches"]},
            "phases_ms": {k: inf[k] for k in ("ms_setup", "ms_lanczos", "ms_eigen", "ms_mu", "ms_extract", "ms_total")},
            "clocks": clk.summary(), "n_colours": nc, "mu": r["mu"], "generation_s": t_gen,
            "trP_minus_ne2": r["trP"] - ne / 2, "workspace_GB": inf["workspace_bytes"] / 1e9}
    gold = ROOT / "tests" / "golden" / "subsample_512.npz"
    if gold.exists():
        gs = np.load(gold)
        line["vs_oracle_512_molecule_subsample"] = {
            "dE_band_eV_per_molecule": 2 * r["trPH"] / n - 2 * float(gs["trPH"]) / int(gs["n_mol"]),
            "dTrP_per_molecule": r["trP"] / n - float(gs["trP"]) / int(gs["n_mol"]),
            "note": "intensive quantities of the 10^6-molecule build against the oracle's on a 512-molecule system "
                    "of the same generator (finite-size and seed spread about 0.05 eV per molecule)"}
    ctx.close()
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "million":
        return run_million(a)
    os.environ.setdefault("CSS_TIMING", "1")
    import torch
    import paper_2605_20918_gb300 as css
    from paper_2605_20918_gb300 import build as cbuild
    from paper_2605_20918_gb300 import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        cbuild.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    prec = {"mixed": css.CSS_MIXED_FP32, "3xtf32": css.CSS_MIXED_3XTF32,
            "fp64-split": css.CSS_FP64_SPLIT}.get(a.precision, css.CSS_FP64)
    mixed = prec in (css.CSS_MIXED_FP32, css.CSS_MIXED_3XTF32)
    from paper_2605_20918_gb300 import shard
    n_steps = a.warmup + a.steps
    my = shard.rank_steps(rank, ws, n_steps)
    geoms = build_inputs(a, my)
    # inputs resident in HBM before the timed region
    dev_in = {}
    for t, (g, H) in geoms.items():
        dev_in[t] = (torch.as_tensor(g.pos, device=dev), css.DeviceBSR.from_host(H, dev))
    g0, H0 = geoms[my[0] % a.geometries]
    colour = torch.empty(a.n_mol, dtype=torch.int32, device=dev)
    sign = torch.empty(a.n_mol * H0.b, dtype=torch.int8, device=dev)
    P = {t: torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev) for t, (g, H) in geoms.items()}
    ctx = css.Context(local)
    stream = torch.cuda.current_stream(dev)
    ne = synth.n_electrons(a.n_mol)

    def step(i):
        t = shard.geometry_of(my[i], a.geometries)
        xyz, Hd = dev_in[t]
        nc = ctx.color(xyz, geoms[t][0].box, a.r_col, 1004, colour)
        ctx.probes(colour, Hd.b, 1005, sign)
        r = ctx.density(Hd, colour, sign, nc, P[t], kT=0.05, n_elec=ne, m=a.m, precision=prec)
        inf = ctx.info()
        return r, nc, inf

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches0 = ctx.info()["kernel_launches"]
    spmm_ms, rows_ms, results = [], [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for i in range(a.warmup, n_steps):
            r, nc, inf = step(i)
            spmm_ms.append(inf["ms_spmm"])
            rows_ms.append(inf["ms_rows"])
            results.append((r, nc, inf))
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = ctx.info()["kernel_launches"] - launches0
    if ws > 1:
        elapsed = shard.max_over_ranks(elapsed, dev)
        dist.barrier()
    value = shard.seconds_per_build(elapsed, a.steps, ws)
    last_r, last_nc, last_inf = results[-1]
    spmm_avg = statistics.mean(spmm_ms)
    rows_avg = statistics.mean(rows_ms)
    achieved = last_inf["spmm_flops"] / (spmm_avg * 1e-3) / 1e12
    pk = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = fp32_peak_tflops(n_sm, pk["sm_max_mhz"])
    tf32_peak = tf32_peak_tflops(pk)
    tc = (os.environ.get("CSS_HV_TC") == "1" or prec == css.CSS_MIXED_3XTF32) and mixed and 16 < H0.b <= 24
    split = prec == css.CSS_FP64_SPLIT
    hv_name, hv_version = hv_kernel(mixed, H0.b, tc)
    if split:
        hv_name, hv_version = ("k_spmm_df (FP64-accurate H*V in FP32 hi + lo pairs on the FP32 FMA pipe)",
                               "k_spmm_df")
    # the split arithmetic takes 11 FP32 lane operations per FP64-equivalent term (2 flop)
    peak = (tf32_peak if tc else fp32_peak) if mixed else (fp32_peak / 11.0 if split else FP64_PEAK)
    traffic = None
    tf = ROOT / "profiles" / "spmm_traffic.json"
    if tf.exists():
        try:
            d = json.loads(tf.read_text())
            if d.get("kernel_version") == hv_version and d.get("precision") == a.precision and \
                    d.get("n_mol") == a.n_mol:
                traffic = d.get("bytes_per_launch")
        except Exception:
            traffic = None
    cfg = workload_config(a)
    cfg["l2"] = l2_note(H0)
    line = {"metric": METRIC, "value": value, "unit": "s/P-build", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": elapsed / a.steps * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if mixed else ("f64 (H*V in f32 pairs)" if split else "f64"),
            "data": "synthetic", "config": cfg,
            "roofline": {"kernel": hv_name,
                         "bound": "tensor" if tc else ("alu" if mixed or split else "alu_fp64"),
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None if tc else traffic,
                         "peak_source": (f"dense TF32 tensor peak: measured sustained BF16 {pk['bf16_sustained']:.0f} "
                                         f"TF/s x 1.1/2.25 ({pk['source']})" if tc else
                                         f"FP32 FFMA (CUDA-core) ceiling: {n_sm} SMs x 128 lanes x 2 flop x "
                                         f"{pk['sm_max_mhz']:.0f} MHz" if mixed else
                                         f"FP32 FFMA ceiling / 11 FP32 operations per FP64-equivalent term "
                                         f"({n_sm} SMs x 128 lanes x 2 flop x {pk['sm_max_mhz']:.0f} MHz / 11)"
                                         if split else FP64_PEAK_NOTE),
                         "frac_vs_tf32_tensor_peak": achieved / tf32_peak if mixed else None,
                         "launch_ms": spmm_avg, "flops_per_launch": last_inf["spmm_flops"],
                         "alg_bytes_per_launch": last_inf["spmm_bytes"]},
            "roofline_rows": row_roofline(a, H0, last_nc, rows_avg, mixed, pk),
            "clocks": clk.summary(), "gpu_launches": int(launches),
            "phases_ms": {k: last_inf[k] for k in ("ms_setup", "ms_lanczos", "ms_eigen", "ms_mu", "ms_extract",
                                                   "ms_total")},
            "n_colours": last_nc, "trP": last_r["trP"], "mu": last_r["mu"]}
    if rank == 0 and not a.no_fp64_compare and mixed:
        # mixed against FP64 on the last geometry (the FP64 path matches the oracle to ~1e-13)
        t = my[n_steps - 1] % a.geometries
        xyz, Hd = dev_in[t]
        nc = ctx.color(xyz, geoms[t][0].box, a.r_col, 1004, colour)
        ctx.probes(colour, Hd.b, 1005, sign)
        P64 = torch.empty_like(P[t])
        # FP64 P builds of the same geometry: one untimed (workspace, tuning), then two timed with
        # CUDA events on the stream (colour + probes + density, as a timed step of the mixed arm)
        ctx.density(Hd, colour, sign, nc, P64, kT=0.05, n_elec=ne, m=a.m, precision=css.CSS_FP64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            nc = ctx.color(xyz, geoms[t][0].box, a.r_col, 1004, colour)
            ctx.probes(colour, Hd.b, 1005, sign)
            r64 = ctx.density(Hd, colour, sign, nc, P64, kT=0.05, n_elec=ne, m=a.m, precision=css.CSS_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 2e3
        inf64 = ctx.info()
        dP = float((P64 - P[t]).abs().max().item())
        # the same FP64 build with the recurrence's H*V in FP32 pairs (CSS_FP64_SPLIT, b = 6 or 23):
        # one untimed, one timed build, its P against the FP64 P
        split = None
        if Hd.b in (6, 23):
            Psp = torch.empty_like(P64)
            ctx.density(Hd, colour, sign, nc, Psp, kT=0.05, n_elec=ne, m=a.m, precision=css.CSS_FP64_SPLIT)
            torch.cuda.synchronize()
            e0.record(stream)
            nc = ctx.color(xyz, geoms[t][0].box, a.r_col, 1004, colour)
            ctx.probes(colour, Hd.b, 1005, sign)
            rsp = ctx.density(Hd, colour, sign, nc, Psp, kT=0.05, n_elec=ne, m=a.m, precision=css.CSS_FP64_SPLIT)
            e1.record(stream)
            torch.cuda.synchronize()
            infs = ctx.info()
            split = {"s_per_pbuild": e0.elapsed_time(e1) / 1e3, "spmm_ms_per_launch": infs["ms_spmm"],
                     "spmm_fp64_equivalent_tflops": infs["spmm_flops"] / (infs["ms_spmm"] * 1e-3) / 1e12
                     if infs["ms_spmm"] > 0 else None,
                     "max_abs_dP_vs_fp64": float((Psp - P64).abs().max().item()),
                     "dTrP_vs_fp64": rsp["trP"] - r64["trP"],
                     "dE_band_eV_per_molecule_vs_fp64": abs(2 * (rsp["trPH"] - r64["trPH"])) / a.n_mol,
                     "note": "CSS_FP64_SPLIT: FP64 vectors, the recurrence's H*V with FP32 hi + lo pairs and "
                             "error-free products on the FP32 FMA pipe"}
            del Psp
        # FP64 at the mixed run's mu: the error of the mixed arithmetic alone, without the
        # change of mu (any mu in the gap satisfies the electron count)
        r64f = ctx.density(Hd, colour, sign, nc, P64, kT=0.05, n_elec=ne, m=a.m, precision=css.CSS_FP64,
                           mu=last_r["mu"], solve_mu=False)
        dPf = float((P64 - P[t]).abs().max().item())
        line["fp64_compare"] = {"fp64_s_per_pbuild": t64, "mixed_s_per_pbuild": value,
                                "fp64_timed_builds": 2, "fp64_spmm_ms_per_launch": inf64["ms_spmm"],
                                "fp64_spmm_tflops": inf64["spmm_flops"] / (inf64["ms_spmm"] * 1e-3) / 1e12
                                if inf64["ms_spmm"] > 0 else None,
                                "speedup_mixed_vs_fp64": t64 / value, "max_abs_dP": dP,
                                "max_abs_dP_same_mu": dPf,
                                "dE_band_eV_per_molecule_same_mu": abs(2 * (last_r["trPH"] - r64f["trPH"])) / a.n_mol,
                                "dE_band_eV_per_molecule": abs(2 * (last_r["trPH"] - r64["trPH"])) / a.n_mol,
                                "dTrP": last_r["trP"] - r64["trP"], "mu_fp64": r64["mu"], "fp64_split": split,
                                "note": "mixed P of the last timed geometry against the FP64 path on the same geometry"}
    if rank == 0 and not a.no_modes:
        # the other matrix functions of the library on the same workload, one build each
        # (after a warm-up call): the energy-weighted density matrix and S^-1/2 of an overlap
        t = my[n_steps - 1] % a.geometries
        xyz, Hd = dev_in[t]
        nc = ctx.color(xyz, geoms[t][0].box, a.r_col, 1004, colour)
        ctx.probes(colour, Hd.b, 1005, sign)
        PE = torch.empty_like(P[t])
        ew = css.CSS_SYMMETRIZE | css.CSS_ENERGY_WEIGHTED
        ctx.density(Hd, colour, sign, nc, PE, kT=0.05, n_elec=ne, m=a.m, precision=prec, flags=ew)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rE = ctx.density(Hd, colour, sign, nc, PE, kT=0.05, n_elec=ne, m=a.m, precision=prec, flags=ew)
        torch.cuda.synchronize()
        tE = time.perf_counter() - t0
        del PE
        S = synth.overlap(geoms[t][0], a.kind)
        Sd = css.DeviceBSR.from_host(S, dev)
        colS = torch.empty(a.n_mol, dtype=torch.int32, device=dev)
        signS = torch.empty(a.n_mol * S.b, dtype=torch.int8, device=dev)
        PS = torch.empty((S.nnzb, S.b, S.b), dtype=torch.float64, device=dev)
        fl = css.CSS_SYMMETRIZE | css.CSS_INV_SQRT
        ncS = ctx.color(xyz, geoms[t][0].box, 9.0, 1004, colS)
        ctx.probes(colS, S.b, 1005, signS)
        ctx.density(Sd, colS, signS, ncS, PS, m=10, precision=prec, flags=fl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ncS = ctx.color(xyz, geoms[t][0].box, 9.0, 1004, colS)
        ctx.probes(colS, S.b, 1005, signS)
        rS = ctx.density(Sd, colS, signS, ncS, PS, m=10, precision=prec, flags=fl)
        torch.cuda.synchronize()
        tS = time.perf_counter() - t0
        Hp = torch.empty_like(P[t])
        ctx.hprime(Sd, Hd, colS, signS, ncS, PS, Hp, m=10, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rH = ctx.hprime(Sd, Hd, colS, signS, ncS, PS, Hp, m=10, precision=prec)
        torch.cuda.synchronize()
        tH = time.perf_counter() - t0
        line["modes"] = {
            "energy_weighted": {"s_per_build": tE, "trace": rE["trP"],
                                "note": "rho_E = f(H) H in each colour's Krylov subspace, same workload"},
            "inv_sqrt_overlap": {"s_per_build": tS, "trace": rS["trP"], "n_colours": int(ncS),
                                 "note": f"S^-1/2 of a synthetic {a.n_mol}-molecule overlap ({S.nnzb} blocks), "
                                         "R_col^S = 9 A, Krylov depth 10, colour + probes + density"},
            "hprime": {"s_per_call": tH, "trace": rH["trHp"],
                       "note": "S~^-1/2 and H' (two-pass Lanczos on S keeping Y, H Y, S~^-1/2 H Y, extraction)"}}
        del PS, Sd, Hp
        # batched serving: 32 systems of uneven size (200-5000 molecules, log-uniform, minimal
        # basis, R_col = 10 A, m = 30) in one css_density_batch call against one call each
        sizes = synth.log_uniform_sizes(32)
        sysd = []
        for i, n_i in enumerate(sizes):
            gi = synth.water_box(int(n_i), seed=1001 + i)
            Hi = synth.hamiltonian(gi, "minimal")
            sysd.append((gi, css.DeviceBSR.from_host(Hi, dev), torch.as_tensor(gi.pos, device=dev),
                         torch.empty(int(n_i), dtype=torch.int32, device=dev),
                         torch.empty(int(n_i) * Hi.b, dtype=torch.int8, device=dev),
                         torch.empty((Hi.nnzb, Hi.b, Hi.b), dtype=torch.float64, device=dev)))

        def batched(p=prec):
            ncs = [ctx.color(x, gi.box, 10.0, 1004, ci) for gi, Hd_i, x, ci, si, Pi in sysd]
            for (gi, Hd_i, x, ci, si, Pi) in sysd:
                ctx.probes(ci, Hd_i.b, 1005, si)
            fs = [{"kT": 0.05, "n_elec": synth.n_electrons(gi.n_mol), "solve_mu": True} for gi, *_ in sysd]
            return ctx.density_batch([d[1] for d in sysd], [d[3] for d in sysd], [d[4] for d in sysd], ncs,
                                     [d[5] for d in sysd], fs, m=30, precision=p)

        def one_by_one():
            for gi, Hd_i, x, ci, si, Pi in sysd:
                nci = ctx.color(x, gi.box, 10.0, 1004, ci)
                ctx.probes(ci, Hd_i.b, 1005, si)
                ctx.density(Hd_i, ci, si, nci, Pi, kT=0.05, n_elec=synth.n_electrons(gi.n_mol), m=30, precision=prec)

        times = {}
        for name, fn in (("batched", batched), ("one_by_one", one_by_one)):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            times[name] = time.perf_counter() - t0
        # the colouring kept across the consecutive geometries held on the device (the first
        # update colours from scratch; its time is not in ms_recolour)
        ts = sorted(dev_in)
        cr = colour_reuse(ctx, [dev_in[t][0] for t in ts], geoms[ts[0]][0].box, a.r_col, colour)
        cr["geometry_indices"] = ts
        cr["note"] = ("css_color_update along the MD-like sequence: keep the colouring while no same-coloured "
                      "pair is closer than R_col, else recolour at R_col + skin")
        line["modes"]["md_colour_reuse"] = cr
        batch = {"batched_s": times["batched"], "one_by_one_s": times["one_by_one"],
                 "molecules": int(sizes.sum()), "sizes_min_max": [int(sizes.min()), int(sizes.max())],
                 "note": "32 systems, 6 orbitals, R_col 10 A, m 30: css_density_batch vs css_density per system"}
        # both precisions side by side against the oracle (stored oracle values of the smallest and
        # the largest system: tests/golden/make_batch_golden.py)
        gold = ROOT / "tests" / "golden" / "batch32_systems.npz"
        if gold.exists():
            gb = np.load(gold)
            for pname, p in (("fp64", css.CSS_FP64), ("mixed", css.CSS_MIXED_FP32)):
                batched(p)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rb = batched(p)
                torch.cuda.synchronize()
                err = {"batched_s": time.perf_counter() - t0}
                for i in gb["systems"]:
                    i = int(i)
                    gi, Pi = sysd[i][0], sysd[i][5]
                    got = Pi[torch.as_tensor(gb[f"blocks_{i}"], device=dev)].cpu().numpy()
                    err[f"system_{i}_{gi.n_mol}_molecules"] = {
                        "max_abs_dP_sampled": float(np.abs(got - gb[f"P_{i}"]).max()),
                        "dE_band_eV_per_molecule": abs(2 * (rb["trPH"][i] - float(gb[f"trPH_{i}"]))) / gi.n_mol,
                        "dTrP": rb["trP"][i] - float(gb[f"trP_{i}"]), "dmu_eV": rb["mu"][i] - float(gb[f"mu_{i}"])}
                batch[pname] = err
            batch["oracle_note"] = ("errors against the oracle's density matrix (mu solved, symmetrised) of the smallest "
                                    "and the largest system: 256 sampled blocks each, Tr(PH) and Tr P")
        line["modes"]["batch_32_systems"] = batch
        del sysd
        line["modes"]["n4096_23_orbitals"] = mode_4096(a, ctx, css, synth, dev, stream)
    if not a.no_e2e:
        # end to end through css_pbuild with host buffers: pinned host inputs in, P out per step
        pin = {}
        for i in range(a.warmup, n_steps):
            t = shard.geometry_of(my[i], a.geometries)
            g, H = geoms[t]
            hv = torch.empty(H.val.shape, dtype=torch.float64, pin_memory=True)
            hv.numpy()[...] = H.val
            pin[t] = (np.ascontiguousarray(g.pos), synth.BSR(H.n_brow, H.b, H.row_ptr, H.col_idx, hv.numpy()),
                      torch.empty(H.val.shape, dtype=torch.float64, pin_memory=True), hv)
        flags = css.CSS_SYMMETRIZE | css.CSS_HOST_IO
        t0s = my[a.warmup] % a.geometries
        ctx.pbuild(pin[t0s][0], geoms[t0s][0].box, pin[t0s][1], pin[t0s][2].numpy(), r_col=a.r_col, kT=0.05,
                   n_elec=ne, m=a.m, precision=prec, flags=flags)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for i in range(a.warmup, n_steps):
            t = shard.geometry_of(my[i], a.geometries)
            pos, Hh, Ph, _ = pin[t]
            ctx.pbuild(pos, geoms[t][0].box, Hh, Ph.numpy(), r_col=a.r_col, kT=0.05, n_elec=ne, m=a.m,
                       precision=prec, flags=flags)
            h2d += pos.nbytes + Hh.row_ptr.nbytes + Hh.col_idx.nbytes + Hh.val.nbytes
            d2h += Ph.numel() * 8
        e2e_t = time.perf_counter() - t0
        if ws > 1:
            e2e_t = shard.max_over_ranks(e2e_t, dev)
        line["e2e"] = {"value": shard.seconds_per_build(e2e_t, a.steps, ws), "unit": "s/P-build", "h2d_bytes_per_step": h2d // a.steps,
                       "d2h_bytes_per_step": d2h // a.steps, "api": "css_pbuild(CSS_HOST_IO)"}
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        g, H = geoms[my[0] % a.geometries]
        line["cpu_baseline"] = cpu_baseline(a, g, H)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
