"""Writes cantilever3d_60x20x4_oc.json: the oracle's trajectory (compliance
and max density change per iteration) of the paper's 3D cantilever (Sec. 5.4)
under Algorithm 1 with the sensitivity filter.  Calls only oracle/ and the
input generators.  Run from the repository root:

    python tests/golden/make_cantilever3d_oc.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2505_02438_gb300 import workloads as W  # noqa: E402


def main():
    wl, fixed, f = W.cantilever_3d_oc(60, 20, 4)
    cen = wl.coords[wl.cells].mean(axis=1)
    vol = np.ones(len(wl.cells))       # unit cubes
    mat = (1.0, 1e-9, 0.3, 3.0, 0)
    x, hist = oracle.oc_loop("hex", 1, wl.coords, wl.cells, mat, fixed, f, 1.5, 0.3, vol, cen,
                             callback=lambda it, h: print(it, h, flush=True))
    out = {"problem": "paper Sec. 5.4: 60x20x4 unit hexahedra, x = 0 fixed, -1 along y on each node of the edge "
                      "x = 60, y = 0; E0 = 1, Emin = 1e-9, nu = 0.3, p = 3, volfrac 0.3, sensitivity filter r = 1.5, "
                      "OC move 0.2, eta 0.5, bisection on [0, 1e9] to 1e-3, stop at max change <= 0.01",
           "c": [h[0] for h in hist], "change": [h[1] for h in hist],
           "final_volume_fraction": float(np.dot(vol, x) / vol.sum())}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cantilever3d_60x20x4_oc.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
