"""Writes tests/golden/bem60k_oracle.json: the FP64 oracle on the n = 60000
BEM-like workload (a_ij = 1/(4 pi |x_i - x_j|), a_ii = sqrt(n), points uniform
on the unit sphere in RCB order, FP32 storage; leaf 512, rtol 1e-6,
d0/d_step 256/128, R seed 1004).  It stands in for the paper's BEM sphere
experiment with adaptive sampling (Section 4, Table 5, n = 58800).

Calls only oracle/ and workloads/.  Records, for the GPU parity test and the
benchmark's CPU baseline:
  * the fingerprint of the FP32 matrix (the GPU builds the same bits);
  * per-node intervals, ranks and the sample count at which each node
    compressed; passes, final sample count, max rank;
  * the oracle's probe error ||(A - H) G||_F / ||A G||_F with 64 probes
    G = numpy default_rng(77) standard normals;
  * the wall time of the full compression and of a bounded sample (the same
    family, schedule and tolerance at n = 12000), with host, cores and BLAS
    threads, so that a shorter run of the sample elsewhere can be scaled.

    python tests/golden/make_bem60k_golden.py [--n N] [--out PATH]

Needs about 40 GB of host memory at n = 60000 and runs for tens of minutes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import hss_oracle as O  # noqa: E402
import workloads as W  # noqa: E402

SPEC = dict(family="bem_like_sphere", n=60000, leaf=512, rtol=1e-6, d0=256, d_step=128,
            point_seed=1003, r_seed=1004, probes=64, probe_seed=77, sample_n=12000)


def bem_fp32(n, leaf, seed):
    pts = W.points_unit_sphere(n, seed)
    pts = pts[W.rcb_order(pts, leaf)]
    return W.bem_like(pts, dtype=np.float32, device="cpu")


def oracle_run(A64, spec):
    t0 = time.perf_counter()
    h = O.compress(A64, spec["rtol"], leaf_size=spec["leaf"], d0=spec["d0"],
                   d_step=spec["d_step"], seed=spec["r_seed"])
    return h, time.perf_counter() - t0


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max(i.get("num_threads", 0) for i in info) if info else None
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=SPEC["n"])
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "bem60k_oracle.json"))
    args = ap.parse_args()
    spec = dict(SPEC, n=args.n)
    n = spec["n"]

    # bounded sample: the same family and settings at n = sample_n
    As = bem_fp32(spec["sample_n"], spec["leaf"], spec["point_seed"]).numpy().astype(np.float64)
    _, t_sample = oracle_run(As, spec)
    del As
    print(f"sample n={spec['sample_n']}: {t_sample:.1f} s", flush=True)

    A32 = bem_fp32(n, spec["leaf"], spec["point_seed"])
    fp = W.fingerprint(A32)
    A64 = A32.numpy().astype(np.float64)
    del A32
    print(f"matrix n={n} built, fingerprint {fp}", flush=True)
    h, t_full = oracle_run(A64, spec)
    print(f"oracle: {t_full:.1f} s, {h.passes} passes, d={h.d}, max rank {h.max_rank()}",
          flush=True)
    G = np.random.default_rng(spec["probe_seed"]).standard_normal((n, spec["probes"]))
    AG = A64 @ G
    HG = O.matvec(h, G)
    e_probe = float(np.linalg.norm(AG - HG) / np.linalg.norm(AG))
    print(f"probe error {e_probe:.3e}", flush=True)
    ranks = h.ranks()
    nodes = [dict(id=nd.id, lo=nd.lo, hi=nd.hi, depth=nd.depth, parent=nd.parent,
                  kr=(ranks[nd.id][0] if nd.id else -1), kc=(ranks[nd.id][1] if nd.id else -1),
                  d_compressed=h.data[nd.id].d_compressed)
             for nd in h.nodes]
    out = dict(spec=spec, fingerprint_fp32=fp, passes=h.passes, d_final=h.d,
               max_rank=h.max_rank(), probe_rel_err=e_probe, nodes=nodes,
               oracle_s=t_full, sample_s=t_sample,
               host=dict(node=platform.node(), machine=platform.machine(),
                         processor=platform.processor(), cores=os.cpu_count(),
                         blas_threads=blas_threads(), numpy=np.__version__),
               note="written by tests/golden/make_bem60k_golden.py (oracle/ and workloads/ only)")
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", args.out, flush=True)


if __name__ == "__main__":
    main()
