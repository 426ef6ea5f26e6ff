"""Golden fixtures: the paper's printed constants and the oracle's regression samples."""
import json
import math
import os

import numpy as np

import oracle as O
from paper_2505_06582_gb300.scenes import SLM, config_scene
from tests.helpers import make_scene

HERE = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_constants_drive_the_oracle():
    c = json.load(open(os.path.join(HERE, "paper_constants.json")))
    assert abs(O.ALPHA_MIN - c["t_eps"]["value"]) < 1e-18
    # Eq. 7: the untilted Gaussian's spectrum at f is 2 pi s^2 exp(-2 pi^2 s^2 f^2) (s in the pair's units)
    s = 3e-5
    slm = SLM(8, 8, 8e-6, 8e-6, (520e-9,))
    U = O.spectrum(make_scene([[0, 0, 0]], [[1, 0, 0, 0]], [[s, s]], [1.0], [[1.0]]), slm)[0]
    fx = 1 / (8 * 8e-6)
    assert abs(U[4, 4].real - c["canonical_pair_constant"]["value"] * s * s) < 1e-15
    expect = c["canonical_pair_constant"]["value"] * s * s * math.exp(-c["canonical_pair_exponent"]["value"] * s * s * fx * fx)
    assert abs(abs(U[4, 5]) - expect) < 1e-12 * expect


def test_oracle_regression_samples():
    g = json.load(open(os.path.join(HERE, "c0_oracle_samples.json")))
    sc, slm = config_scene("c0_plain_fp64")
    vals = O.spectrum_at(sc, slm, np.zeros(len(g["rows"]), np.int32), g["rows"], g["cols"])
    ref = np.array(g["spectrum_re"]) + 1j * np.array(g["spectrum_im"])
    assert np.allclose(vals, ref, rtol=1e-12, atol=1e-22)
    assert np.allclose(O.transmittance(sc)[:16], g["transmittance_first16"], rtol=1e-13, atol=0)
