#!/usr/bin/env python3
"""Write the oracle's results for the large parity cases to tests/golden/oracle_<case>.json.

The GPU tests at 20,000 and 150,000 points compare against these stored values, because the FP64
oracle needs minutes per case on a host's cores.  This script calls only the oracle (and the seeded
input generators); nothing here comes from the CUDA path.  Each file records the inputs'
checksums, so a test can confirm that its machine generated the same X and y, and the exact
hyperparameters used.

    python tests/golden/make_oracle_large.py [case ...]     # default: every case

Cases (Sec. 3 LML, SLQ log-determinant and Hutchinson gradient with identical Rademacher probes):
  clusters_3d_20k_t{0..7}  20,000 points of the clustered 3-D generator (100 entries per row),
                           L = 8 (42 parameters), 8 hyperparameter sets drawn around the base one,
                           64 probes x 100 steps
  clusters_3d_150k_t{0,1}  150,000 points of the same generator, the base and one drawn set
  sphere_4d_150k           150,000 points of the 4-D sphere x time x elevation generator
                           (60 entries per row), 32 probes x 100 steps
  sphere_4d_10m            the full 10,000,000-point workload of that generator (about 600 M stored
                           entries; the oracle's CG to 1e-8), 32 probes x 100 steps
  batch0_p{100,32,116}     three problems of the 256-problem batch (the largest, the densest rows,
                           the largest 1-D one), 16 probes x 100 steps, LML only
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_06143_gb300 import workloads as W  # noqa: E402

CG_TOL = 1e-9


def cases():
    out = {}
    for k in range(8):
        out[f"clusters_3d_20k_t{k}"] = dict(workload="clusters_3d", n=20000, target=100.0, theta_set=100,
                                            theta_index=k, probes=64, steps=100, seed=0)
    out["clusters_3d_150k_t0"] = dict(workload="clusters_3d", n=150000, target=100.0, theta_set=None,
                                      theta_index=0, probes=64, steps=100, seed=0)
    out["clusters_3d_150k_t1"] = dict(workload="clusters_3d", n=150000, target=100.0, theta_set=101,
                                      theta_index=0, probes=64, steps=100, seed=0)
    out["sphere_4d_150k"] = dict(workload="sphere_4d", n=150000, target=60.0, theta_set=None,
                                 theta_index=0, probes=32, steps=100, seed=0)
    out["sphere_4d_10m"] = dict(workload="sphere_4d", n=10_000_000, target=60.0, theta_set=None,
                                theta_index=0, probes=32, steps=100, seed=0, cg_tol=1e-8)
    # problems of the 256-problem batch (seed 0): the largest, the densest rows, the largest 1-D
    for idx in (100, 32, 116):
        out[f"batch0_p{idx}"] = dict(workload="batch", n=None, target=None, theta_set=None, theta_index=idx,
                                     probes=16, steps=100, seed=0, grad=False)
    return out


def inputs(spec):
    """X, y and the hyperparameter dict of a case (the same calls the GPU tests make)."""
    if spec["workload"] == "batch":
        w = W.batch(0)[spec["theta_index"]]
        return w["X"], w["y"], w["hyper"]
    gen = {"clusters_3d": W.clusters_3d, "sphere_4d": W.sphere_4d}[spec["workload"]]
    w = gen(0, n=spec["n"], target_nnz=spec["target"])
    hyper = w["hyper"]
    if spec["theta_set"] is not None:
        hyper = W.perturbed_hypers(hyper, spec["theta_index"] + 1, spec["theta_set"])[spec["theta_index"]]
    return w["X"], w["y"], hyper


def run(name, spec):
    X, y, hyper = inputs(spec)
    h = oracle.Hyper(**hyper)
    t0 = time.time()
    tol = spec.get("cg_tol", CG_TOL)
    want_grad = spec.get("grad", True)
    s = oracle.lml_slq(X, y, h, m=spec["probes"], k=spec["steps"], seed=spec["seed"], tol=tol, grad=want_grad)
    rec = {
        "case": name, **spec, "cg_tol": tol, "oracle_threads": oracle.num_threads(),
        "oracle_seconds": round(time.time() - t0, 1),
        "checksums": W.checksums(X, y),
        "hyper": {"d": hyper["d"], "r": hyper["r"], "sigma2": hyper["sigma2"], "beta": hyper["beta"],
                  "w0": hyper["w0"], "kind": hyper["kind"], "centers": np.asarray(hyper["centers"]).tolist(),
                  "radii": np.asarray(hyper["radii"]).tolist(), "amps": np.asarray(hyper["amps"]).tolist()},
        "nnz": int(s["csr"].nnz), "lml": s["lml"], "quad": s["quad"], "logdet": s["logdet"],
        "logdet_diag": s["logdet_diag"], "relres": s["relres"],
        "probe_quadrature_std": float(np.std(s["probe_quadrature"], ddof=1)),
        "grad": [float(v) for v in s["grad"]] if want_grad else None,
        "n_points": int(X.shape[0]),
    }
    path = os.path.join(HERE, f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"{name}: {rec['oracle_seconds']} s, nnz {rec['nnz']}, lml {rec['lml']:.12g}", flush=True)


def main():
    oracle.build()
    want = sys.argv[1:] or list(cases())
    for name in want:
        run(name, cases()[name])


if __name__ == "__main__":
    main()
