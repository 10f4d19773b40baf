"""Write ``fc_<kind>_L4096.json``: the finite-size critical force at L = 4096 of the random-field
chain (R ~ N(0,1), linear interpolation; ``rf``) or of the Gaussian random-bond chain with a
linear spline (Case 3 of Sec. IV.C; ``rbg_linear``) or a Catmull-Rom spline (Case 1;
``rbg_cubic``), found by bisection with the CPU oracle only.

Criterion (the short-time-dynamics bracketing of Sec. III.A, made concrete): relax 8 samples
from the flat start to t = 500 and fit the log-log slope of V(t) t^{beta/nu z} over the last
decade of t, with beta/nu z = 0.128 (Sec. IV.E).  A positive slope means V saturates (f above
f_c), a negative one that V decays faster than the critical power law (f below f_c).

Run: python tests/golden/make_fc_oracle.py rf|rbg_linear|rbg_cubic   (about a minute each on 8 cores)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from qew_workloads import SEED, log_spaced_steps  # noqa: E402

L, N_SAMPLES, DT, N_STEPS, BETA_NU_Z = 4096, 8, 0.1, 5000, 0.128
KINDS = {"rf": ("RF", oracle.KIND_RF), "rbg_linear": ("RB Gaussian, linear spline", oracle.KIND_RBG_LINEAR),
         "rbg_cubic": ("RB Gaussian, Catmull-Rom spline", oracle.KIND_RBG_CUBIC)}


def drift(f: float, kind: int) -> float:
    steps = log_spaced_steps(N_STEPS, 30, include_zero=False)
    out = oracle.run([L] * N_SAMPLES, f, DT, kind, SEED, steps)
    V = out["v"].mean(axis=1)
    t = steps * DT
    sel = t >= t[-1] / 10
    if np.any(V[sel] <= 0):
        return -np.inf
    return float(np.polyfit(np.log(t[sel]), np.log(V[sel] * t[sel] ** BETA_NU_Z), 1)[0])


def main() -> None:
    name = sys.argv[1] if len(sys.argv) > 1 else "rf"
    label, kind = KINDS[name]
    lo, hi = 0.5, 3.0
    history = []
    for _ in range(14):
        mid = 0.5 * (lo + hi)
        d = drift(mid, kind)
        history.append((mid, d))
        if d >= 0:
            hi = mid
        else:
            lo = mid
    fc = 0.5 * (lo + hi)
    rec = {
        "L": L, "samples": N_SAMPLES, "dt": DT, "n_steps": N_STEPS, "seed": SEED, "kind": label,
        "beta_over_nu_z": BETA_NU_Z, "bracket": [lo, hi], "f_c": fc,
        "history": history,
        "_cite": "bracketing criterion of Sec. III.A; exponent ratio of Sec. IV.E",
        "_made_by": f"tests/golden/make_fc_oracle.py {name} (CPU oracle only)",
    }
    with open(os.path.join(HERE, f"fc_{name}_L4096.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps({"f_c": fc, "bracket": [lo, hi]}))


if __name__ == "__main__":
    main()
