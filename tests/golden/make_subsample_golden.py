"""Write tests/golden/subsample_512.npz: the oracle's Tr P, Tr(PH) and mu of the 512-molecule,
6-orbital system built by the same generator as the 10^6-molecule workload (R_col = 10 A, m = 30,
kT = 0.05 eV, mu solved), the reference for the per-molecule band energy and electron count of
the benchmark's 10^6-molecule run.

Only the oracle (oracle/) and the seeded input generator (synth) are called.

Usage: python tests/golden/make_subsample_golden.py   (seconds)
"""
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2605_20918_gb300 import synth  # noqa: E402


def main():
    g = synth.water_box(512)
    H = synth.hamiltonian(g, "minimal")
    col, nc = oracle.color(g.pos, g.box, 10.0, 1004)
    ref = oracle.density(H, col, oracle.probes(col, H.b, 1005), nc, kT=0.05, n_elec=synth.n_electrons(512), m=30)
    np.savez_compressed(Path(__file__).with_name("subsample_512.npz"), n_mol=512, trP=ref["trP"], trPH=ref["trPH"],
                        mu=ref["mu"], n_colours=nc)
    print(ref["trP"], ref["trPH"], ref["mu"], nc)


if __name__ == "__main__":
    main()
