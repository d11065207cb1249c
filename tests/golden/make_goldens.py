"""Write tests/golden/workloads.json: expected counts of the full-size seeded
workloads, computed by the CPU oracle only (graphgen builds the inputs,
oracle/ computes every value; nothing here touches the CUDA path).

    python tests/golden/make_goldens.py [--threads N]

Values and the tier that produced them:
  er-10k      triangle                       O2 nested-loop plan (full)
  rmat22      triangle, 4-clique              O2 nested-loop plan (full, OpenMP)
  chunglu-1m  triangle, diamond, 4-cycle,     O3 closed forms (Section 5.4
              tailed-triangle, 3-star,        decompositions: per-edge
              4-path, wedge (edge-induced)    triangle counts, co-degrees)
The 5-clique count of rmat22 is not stored: the O2 plan would need hours of
CPU time; the GPU result is checked on sampled task ranges instead.
Each workload also stores the FNV-1a checksum of its CSR so that a test can
confirm that another host generated the identical graph.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    out = {}
    t0 = time.time()
    g = gg.workload("er-10k")
    out["er-10k"] = {"checksum": gg.csr_checksum(g), "n": g.n, "edges": g.m,
                     "counts": {"triangle": O.count(g, "triangle")},
                     "method": {"triangle": "O2"}}
    print("er-10k", out["er-10k"], time.time() - t0, flush=True)

    g = gg.workload("rmat22")
    out["rmat22"] = {"checksum": gg.csr_checksum(g), "n": g.n, "edges": g.m,
                     "counts": {"triangle": O.count(g, "triangle", nthreads=args.threads),
                                "4-clique": O.count(g, "4-clique", nthreads=args.threads)},
                     "method": {"triangle": "O2", "4-clique": "O2"}}
    print("rmat22", out["rmat22"], time.time() - t0, flush=True)

    g = gg.workload("chunglu-1m")
    ids = O.identities(g, nthreads=args.threads)
    out["chunglu-1m"] = {"checksum": gg.csr_checksum(g), "n": g.n, "edges": g.m,
                         "counts": {"triangle": ids["triangle"], "diamond": ids["diamond_e"],
                                    "4-cycle": ids["4-cycle_e"],
                                    "tailed-triangle": ids["tailed-triangle_e"],
                                    "3-star": ids["3-star_e"], "4-path": ids["4-path_e"],
                                    "wedge": ids["wedge_e"]},
                         "method": {k: "O3" for k in ["triangle", "diamond", "4-cycle",
                                                      "tailed-triangle", "3-star", "4-path",
                                                      "wedge"]}}
    print("chunglu-1m", out["chunglu-1m"], time.time() - t0, flush=True)
    with open(os.path.join(HERE, "workloads.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
