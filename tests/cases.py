"""Shared test configuration: one dict describes a case; these helpers build
the oracle's Config and the CUDA library's Params from it, and measure the
normwise per-field error used as the parity metric:
    e_f = max|gpu - cpu| / max(max|cpu_f|, 1e-3 max_g max|cpu_g|)
(the floor keeps fields whose exact value is ~0 from dividing by rounding),
and the rounding-aware form of the float64 right-hand-side bar (see
rounding_aware_errors)."""
import math

import numpy as np

import oracle as O


def oracle_cfg(c):
    return O.Config(n=c["n"], xmin=c["xmin"], h=c["h"], periodic=c.get("boundary", "periodic") == "periodic",
                    use_w=c.get("conformal", "W") == "W", slicing=c.get("slicing", "1+log"),
                    shift=c.get("shift", "gamma-driver"), eta=c.get("eta", 2.0), q_R=c.get("q_R", math.inf),
                    ko_eps=c.get("ko_eps", 0.1), dt=c.get("dt", 0.25 * c["h"]),
                    w_floor=c.get("w_floor", 1e-10), r_excise=c.get("r_excise", 1.0),
                    punctures=c.get("punctures", []))


def gpu_params(c):
    from paper_1111_3344_gb300.bssn import Params
    return Params(n=tuple(c["n"]), xmin=tuple(c["xmin"]), h=c["h"], boundary=c.get("boundary", "periodic"),
                  conformal=c.get("conformal", "W"), slicing=c.get("slicing", "1+log"),
                  shift=c.get("shift", "gamma-driver"), eta=c.get("eta", 2.0), q_R=c.get("q_R", math.inf),
                  ko_eps=c.get("ko_eps", 0.1), dt=c.get("dt", 0.25 * c["h"]),
                  precision=c.get("precision", "fp64"), w_fp64_threshold=c.get("w_fp64_threshold", 0.0),
                  r_excise=c.get("r_excise", 1.0), w_floor=c.get("w_floor", 1e-10))


def bl_params(c):
    p = [len(c["punctures"])]
    for q in c["punctures"]:
        p += list(q)
    return p


def normwise_errors(gpu, cpu):
    gpu = np.asarray(gpu).reshape(gpu.shape[0], -1)
    cpu = np.asarray(cpu).reshape(cpu.shape[0], -1)
    fmax = np.abs(cpu).max(axis=1)
    floor = 1e-3 * fmax.max()
    return np.abs(gpu - cpu).max(axis=1) / np.maximum(np.maximum(fmax, floor), 1e-300)


def rounding_aware_errors(gpu, cpu, mag, rtol=1e-12):
    """Per field f, the largest ratio over points p of
        |gpu_pf - cpu_pf| / (rtol max(S_f, M_pf)),
    with S_f the normwise scale of normwise_errors and M_pf the oracle's
    magnitude of the same expression evaluated on absolute values (the
    instrumented oracle build).  A ratio <= 1 passes.

    Where a right-hand side is a small difference of much larger terms (K and
    At half a cell from a puncture: W^2 times the lapse Laplacian against
    2 W^2 grad(phi).grad(alpha)), two float64 evaluations in different orders
    differ by a few u M_pf, u = 2^-53, which can exceed 1e-12 of the field's
    largest value; elsewhere M_pf is small and the bar is the normwise
    1e-12 S_f.  Arrays are (24, ...) with the field axis first."""
    gpu = np.asarray(gpu).reshape(gpu.shape[0], -1)
    cpu = np.asarray(cpu).reshape(cpu.shape[0], -1)
    mag = np.asarray(mag).reshape(mag.shape[0], -1)
    fmax = np.abs(cpu).max(axis=1)
    scale = np.maximum(np.maximum(fmax, 1e-3 * fmax.max()), 1e-300)
    bar = rtol * np.maximum(scale[:, None], mag)
    return (np.abs(gpu - cpu) / bar).max(axis=1)
