"""Write the stored oracle digests of the full-size clustered workloads.

Runs the exact CPU oracle (``oracle/``, bucketed mode, Method A.6) on
  - the 4,194,304-site Gaussian-mixture workload (``gauss_4m.json``): a
    digest per chunk of 65,536 cells, the totals, and the cells the oracle
    marks degenerate (a vertex with more than three equidistant sites);
  - every set of the 4,096-set batch (``batch_4096.json``): a digest per set;
  - every request of a 200-request serving stream of log-uniform size in
    [100, 10^6], half uniform and half clustered (``serve_stream.json``): a
    digest per request;
and writes the digests (``tests/parity.py``: edge counts, canonical edge
labels, Delaunay pairs) with the digest of each input.  Nothing here runs or
reads the CUDA library: the stored values come from the oracle alone.

Method A.6 takes any bucket side s > 0 and any integer beta > 0, and
Proposition A.8 shows that its endpoint is the exact first hit for every such
choice; eqs. (8.1)-(8.7) fix beta only to bound the expected number of
comparisons for uniform sites.  The digests use the bucket side of Remark
B.1(iv) and beta = 1, which on clustered sites is several times faster than
the beta of eq. (8.7) (the rectangular lists of Step 5 cover fewer crowded
buckets); tests/test_oracle_pins.py checks that beta = 1 returns the same
cells as plain mode and as the default beta.

Usage:  python tests/golden/make_digests.py [gauss_4m] [batch_4096] [serve_stream]
(hours of CPU for all three; each file is written when its workload is done).
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE)):
    if p not in sys.path:
        sys.path.insert(0, p)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from parity import DIGEST_CHUNK, cells_digest, chunk_digests, input_digest  # noqa: E402

BOX = synth.WORLD
BETA = 1
SERVE_REQUESTS = 200
SERVE_SEED = synth.SEED_BASE + 60


def _oracle(xy):
    return oracle.cells(xy, BOX, "bucketed", beta=BETA)


def _write(name, doc):
    path = os.path.join(HERE, name)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=0)
        f.write("\n")
    os.replace(tmp, path)
    print("wrote", path, flush=True)


def _oracle_doc():
    return {"mode": "bucketed (Method A.6)", "bucket_side": "Remark B.1(iv)", "beta": BETA,
            "script": "tests/golden/make_digests.py"}


def gauss_4m():
    xy = synth.workload("gauss_4m")
    n = xy.shape[0]
    t0 = time.time()
    r = _oracle(xy)
    dt = time.time() - t0
    degenerate = np.nonzero(r["stats"][:, 5] > 0)[0]
    _write("gauss_4m.json", {
        "workload": "gauss_4m", "n": int(n), "input_sha256": input_digest(xy),
        "oracle": _oracle_doc(), "oracle_seconds": round(dt, 1),
        "threads": os.cpu_count(), "chunk": DIGEST_CHUNK,
        "n_edges": int(r["labels"].shape[0]), "n_del": int(r["delaunay"].shape[0]),
        "degenerate_cells": [int(k) for k in degenerate],
        "chunks": chunk_digests(r["cell_ptr"], r["labels"], r["delaunay"], n),
    })


def batch_4096():
    xy, ptr = synth.batch_workload()
    S = ptr.shape[0] - 1
    digests = []
    t0 = time.time()
    for j in range(S):
        s = xy[ptr[j]:ptr[j + 1]]
        r = _oracle(s)
        digests.append(cells_digest(r["cell_ptr"], r["labels"], r["delaunay"], 0, s.shape[0]))
        if j % 256 == 255:
            print(f"batch set {j + 1}/{S} {time.time() - t0:.0f} s", flush=True)
    _write("batch_4096.json", {
        "workload": "batch_4096", "n_sets": int(S), "n_sites": int(ptr[-1]),
        "input_sha256": input_digest(xy), "set_ptr_sha256": input_digest(ptr.astype(np.int32)),
        "oracle": _oracle_doc(), "oracle_seconds": round(time.time() - t0, 1),
        "threads": os.cpu_count(), "sets": digests,
    })


def serve_stream_requests():
    """The requests of the stored serving stream: (sizes, kinds, sites)."""
    pools = synth.serve_pools()
    _, sizes, kinds = synth.poisson_requests(SERVE_REQUESTS, 1.0, seed=SERVE_SEED)
    reqs = [synth.serve_request(j + SERVE_SEED * 100000, int(s), int(k), pools)
            for j, (s, k) in enumerate(zip(sizes, kinds))]
    return sizes, kinds, reqs


def serve_stream():
    sizes, kinds, reqs = serve_stream_requests()
    digests, inputs = [], []
    t0 = time.time()
    for j, xy in enumerate(reqs):
        r = _oracle(xy)
        digests.append(cells_digest(r["cell_ptr"], r["labels"], r["delaunay"], 0, xy.shape[0]))
        inputs.append(input_digest(xy)[:32])
        if j % 20 == 19:
            print(f"serve request {j + 1}/{len(reqs)} {time.time() - t0:.0f} s", flush=True)
    _write("serve_stream.json", {
        "workload": "serve_stream", "n_requests": len(reqs), "seed": SERVE_SEED,
        "sizes": [int(s) for s in sizes], "kinds": [int(k) for k in kinds],
        "n_sites": int(sum(int(s) for s in sizes)), "inputs": inputs,
        "oracle": _oracle_doc(), "oracle_seconds": round(time.time() - t0, 1),
        "threads": os.cpu_count(), "requests": digests,
    })


JOBS = {"gauss_4m": gauss_4m, "batch_4096": batch_4096, "serve_stream": serve_stream}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(JOBS)):
        JOBS[name]()
