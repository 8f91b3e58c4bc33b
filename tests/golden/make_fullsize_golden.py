"""Write tests/golden/fullsize_10k_colours.npz (and, with --n-mol 4096, fullsize_4096_colours.npz):
the oracle's unsymmetrised density-matrix columns of two colours of the 10,000-molecule (or
4,096-molecule) 23-orbital workload (R_col = 10 A, m = 40, kT = 0.05 eV), at a fixed chemical
potential, for the full-size GPU parity tests and the benchmark's error report.

Only the oracle (oracle/) and the seeded input generator (synth) are called: the stored values
never come from the CUDA path.  The columns of a colour c are the blocks P~_IJ with colour(J) = c
(Eq. 2 and Eq. 6: P~_IJ = [Q_c Z_c]_I diag(s_J)); each is a full block-Lanczos of depth 40 on the
230,000-row matrix plus its exact diagonalisation, so the oracle needs minutes per colour.

mu is fixed at -4.0 eV, the middle of the gap between the on-site level ranges of the 23-orbital
generator (occupied levels in [-25, -10] eV, virtual ones in [+2, +30] eV).

Usage: python tests/golden/make_fullsize_golden.py [--n-mol 4096]   (about 20 minutes on 8 cores
for 10,000 molecules)
"""
import argparse
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2605_20918_gb300 import synth  # noqa: E402

N_MOL, R_COL, M, KT, MU = 10000, 10.0, 40, 0.05, -4.0
SAMPLES = 32  # stored blocks per colour (seeded choice); the partial traces cover every block


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-mol", type=int, default=N_MOL)
    n_mol = ap.parse_args().n_mol
    t0 = time.time()
    g = synth.water_box(n_mol)
    H = synth.hamiltonian(g, "dzp")
    col, nc = oracle.color(g.pos, g.box, R_COL, 1004)
    sign = oracle.probes(col, H.b, 1005)
    colours = [0, nc - 1]
    out = {"mu": MU, "kT": KT, "m": M, "n_colours": nc, "colours": np.array(colours, np.int32),
           "colour_checksum": np.int64((col.astype(np.int64) * np.arange(n_mol, dtype=np.int64)).sum())}
    rng = np.random.default_rng(2605)
    for c in colours:
        ref = oracle.density(H, col, sign, nc, mu=MU, kT=KT, solve_mu=False, m=M, flags=0, colour_subset=[c])
        blocks = np.nonzero(col[H.col_idx] == c)[0]
        pick = np.sort(rng.choice(blocks, size=min(SAMPLES, blocks.size), replace=False))
        out[f"blocks_{c}"] = pick.astype(np.int64)
        out[f"P_{c}"] = ref["P"][pick]
        out[f"trP_{c}"] = ref["trP"]
        out[f"trPH_{c}"] = ref["trPH"]
        out[f"nblocks_{c}"] = blocks.size
        print(f"colour {c}: {blocks.size} blocks, trP {ref['trP']:.12f} trPH {ref['trPH']:.12f} "
              f"({time.time() - t0:.0f} s)", flush=True)
    name = "fullsize_10k_colours.npz" if n_mol == 10000 else f"fullsize_{n_mol}_colours.npz"
    np.savez_compressed(Path(__file__).with_name(name), **out)


if __name__ == "__main__":
    main()
