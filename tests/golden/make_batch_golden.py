"""Write tests/golden/batch32_systems.npz: the oracle's density matrices of the smallest and the
largest of the 32 batched-serving systems (6 orbitals, 200-5,000 molecules drawn log-uniform,
R_col = 10 A, m = 30, kT = 0.05 eV, mu solved by the oracle's rule, symmetrised), as sampled blocks
plus Tr P, Tr(PH) and mu, for the benchmark's error report of the batched workload.

Only the oracle (oracle/) and the seeded input generator (synth) are called.

Usage: python tests/golden/make_batch_golden.py   (about a minute on 8 cores)
"""
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2605_20918_gb300 import synth  # noqa: E402

R_COL, M, KT = 10.0, 30, 0.05
SAMPLES = 256


def main():
    sizes = synth.log_uniform_sizes(32)
    order = np.argsort(sizes)
    out = {"sizes": sizes, "m": M, "kT": KT, "systems": np.array([order[0], order[-1]], np.int32)}
    rng = np.random.default_rng(32)
    for i in (int(order[0]), int(order[-1])):
        g = synth.water_box(int(sizes[i]), seed=1001 + i)
        H = synth.hamiltonian(g, "minimal")
        col, nc = oracle.color(g.pos, g.box, R_COL, 1004)
        sign = oracle.probes(col, H.b, 1005)
        ref = oracle.density(H, col, sign, nc, kT=KT, n_elec=synth.n_electrons(g.n_mol), m=M)
        pick = np.sort(rng.choice(H.nnzb, size=min(SAMPLES, H.nnzb), replace=False))
        out[f"blocks_{i}"] = pick.astype(np.int64)
        out[f"P_{i}"] = ref["P"][pick]
        out[f"trP_{i}"] = ref["trP"]
        out[f"trPH_{i}"] = ref["trPH"]
        out[f"mu_{i}"] = ref["mu"]
        out[f"n_colours_{i}"] = nc
        print(f"system {i}: {g.n_mol} molecules, {nc} colours, trP {ref['trP']:.9f} mu {ref['mu']:.9f}", flush=True)
    np.savez_compressed(Path(__file__).with_name("batch32_systems.npz"), **out)


if __name__ == "__main__":
    main()
