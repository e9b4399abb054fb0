"""Write the stored exact values under tests/golden/ (calls only the oracle).

    python tests/golden/make_golden.py

dos_fm_L8.json: exact density of states g(E) of the 8x8 periodic Ising
ferromagnet from the oracle's transfer matrix (about 30 s).  The tests pin it
against Kaufman's closed form and use it as the exact reference for E and C.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    L = 8
    Jr, Jd = oracle.couplings(L, 0, 1, 0)
    g = oracle.dos_transfer(L, Jr, Jd)
    N = L * L
    dos = {str(2 * n - 2 * N): str(v) for n, v in enumerate(g) if v}
    with open(os.path.join(HERE, "dos_fm_L8.json"), "w") as f:
        json.dump({"_source": "oracle.dos_transfer(8, FM couplings), written by make_golden.py",
                   "L": L, "g_by_E": dos}, f, indent=1)


if __name__ == "__main__":
    main()
