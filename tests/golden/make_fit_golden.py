"""Writes the stored oracle fits used by the full-size fit-parity tests.

The oracle (plain FP64 C, dual-number gradients, damped Newton to EDM < 1e-12) fits the
seeded Poisson data of a named workload from theta_true; the result, with a fingerprint of
the data it was fitted to, goes to tests/golden/fit_<name>.json.  Only the oracle and the
seeded input generator are called here; a full multivariate fit takes a few minutes on the
host cores, which is why the GPU tests read the stored result instead of refitting.

  python tests/golden/make_fit_golden.py multivariate plain
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1805_11125_gb300 import inputs as I  # noqa: E402


def fingerprint(counts: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(counts, dtype=np.float64).tobytes()).hexdigest()


def dataset(name: str, seed: int = 0):
    s = I.config(name)
    return s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), seed))


def main(names):
    for name in names:
        s = dataset(name)
        t0 = time.time()
        r = O.fit(s, s.theta_true, tol_edm=1e-12)
        sig = np.sqrt(np.maximum(np.diag(r["cov"]), 0.0))
        out = {"config": name, "data_seed": 0, "start": "theta_true",
               "counts_sha256": fingerprint(s.counts_vector()), "counts_sum": float(s.counts_vector().sum()),
               "theta": r["theta"].tolist(), "nll": r["nll"], "sigma": sig.tolist(), "edm": r["edm"],
               "iters": r["iters"], "status": r["status"], "free": s.default_free().tolist(),
               "fit_s": time.time() - t0, "writer": "tests/golden/make_fit_golden.py (oracle only)"}
        with open(os.path.join(HERE, f"fit_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, r["status"], r["iters"], r["nll"], f"{time.time() - t0:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["multivariate", "plain"])
