"""Writes the oracle regression fixtures in this folder.  Calls only ``oracle/``.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2505_06582_gb300.scenes import config_scene  # noqa: E402


def main():
    sc, slm = config_scene("c0_plain_fp64")
    rng = np.random.default_rng(123)
    rows = rng.integers(0, slm.H, 32)
    cols = rng.integers(0, slm.W, 32)
    lam = np.zeros(32, dtype=np.int32)
    vals = O.spectrum_at(sc, slm, lam, rows, cols)
    T = O.transmittance(sc)
    out = {
        "workload": "64 Gaussians, 128x128, 8 um, 520 nm (seed 0, uniform scene)",
        "written_by": "tests/golden/make_golden.py (oracle only)",
        "rows": rows.tolist(), "cols": cols.tolist(),
        "spectrum_re": vals.real.tolist(), "spectrum_im": vals.imag.tolist(),
        "transmittance_first16": T[:16].tolist(),
    }
    with open(os.path.join(os.path.dirname(__file__), "c0_oracle_samples.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
