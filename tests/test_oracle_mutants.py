"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/vor_oracle.c``, plants one plausible mistake (a
dropped term, a flipped sign, a swapped tie rule, a wrong side constant, an
off-by-one window), compiles the copy on the CPU and runs a small set of the
pins against it.  The real oracle is never modified.
"""

import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from bruteforce import halfplane_cell, restricted_delaunay

SRC = os.path.join(os.path.dirname(oracle.__file__), "vor_oracle.c")

MUTANTS = {
    "dropped_term_in_N": ("*Nx = a->c * b->ny - b->c * a->ny;", "*Nx = a->c * b->ny;"),
    "wedge_sign": ("int inw = sg * crossd(t1, N) >= 0 && sg * crossd(N, t2) >= 0;",
                   "int inw = sg * crossd(t1, N) >= 0 && sg * crossd(N, t2) <= 0;"),
    # Remark A.4 ignored: any tied site instead of an extreme one
    "tie_rule_not_extreme": ("    e->ccw = best_ccw.label;\n    e->cw = best_cw.label;",
                             "    e->ccw = ties[nt - 1];\n    e->cw = ties[nt - 1];"),
    "side_constant": ("L.c = 2 * (L.nx * L.nx + L.ny * L.ny);",
                      "L.c = (L.nx * L.nx + L.ny * L.ny);"),
    "open_cell": ("return lhs > rhs ? 1 : (lhs == rhs ? 0 : -1);",
                  "return lhs >= rhs ? 1 : (lhs == rhs ? 0 : -1);"),
    "transposed_right_side": ("case SIDE_RIGHT:  L.nx = w->W - px; L.ny = 0; break;",
                              "case SIDE_RIGHT:  L.nx = w->H - px; L.ny = 0; break;"),
    "window_off_by_one": ("b.x1 = (i64)floordiv128(yhi_x + rup, w->s);",
                          "b.x1 = (i64)floordiv128(yhi_x + rup, w->s) - 1;"),
    # theta_3 := -phi (outside the wedge) for parallel lines
    "parallel_direction": ("t3.x = -l1.ny; t3.y = l1.nx;\n            if (!in_wedge(t1, t2, t3)) { t3.x = -t3.x; t3.y = -t3.y; }",
                           "t3.x = l1.ny; t3.y = -l1.nx;"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(path), "-lm"])
    return str(so)


def _pins_pass() -> bool:
    """A compact subset of the pins; False as soon as one fails."""
    try:
        cases = [(synth.uniform_sites(12, seed=s, box=64), 64) for s in range(4)]
        cases += [(synth.uniform_sites(15, seed=50 + s, box=4096), 4096) for s in range(4)]
        cases.append((synth.lattice_sites(4, 16, 8), 64))
        cases.append((np.array([[100, 400], [300, 400], [500, 400]], dtype=np.int32), 600))
        cases.append((np.array([[30, 50], [70, 20]], dtype=np.int32), (100, 60)))
        # a ray of the projector meets a vertex with three equidistant sites
        cases.append((np.array([[50, 50], [60, 60], [40, 60], [50, 70]], dtype=np.int32), 100))
        for xy, box in cases:
            W, H = (box, box) if np.isscalar(box) else box
            for mode in ("plain", "bucketed"):
                r = oracle.cells(xy, (W, H), mode, bucket_side=max(1, W // 6), beta=1)
                st = r["stats"]
                # counting lemmas of Section 8 / Appendix 3
                if not (np.all(st[:, 0] <= st[:, 6] + 1) and np.all(st[:, 1] <= 2 * st[:, 6])
                        and np.all(st[:, 7] == 0)):
                    return False
                for k in range(len(xy)):
                    a, b = r["cell_ptr"][k], r["cell_ptr"][k + 1]
                    got = ([int(v) for v in r["labels"][a:b]], oracle.vertices_exact(r, k))
                    if got != halfplane_cell(xy, k, W, H):
                        return False
                if W == H:
                    if sorted(map(tuple, r["delaunay"].tolist())) != restricted_delaunay(xy, W, H):
                        return False
        # bucketed vs plain on a larger uniform set
        xy = synth.uniform_sites(3000, seed=3)
        a = oracle.cells(xy, 1 << 20, "bucketed", bucket_side=1 << 15, beta=1)
        b = oracle.cells(xy, 1 << 20, "plain", sel=np.arange(0, 3000, 7))
        for i, k in enumerate(range(0, 3000, 7)):
            la = a["labels"][a["cell_ptr"][k]:a["cell_ptr"][k + 1]].tolist()
            lb = b["labels"][b["cell_ptr"][i]:b["cell_ptr"][i + 1]].tolist()
            if la != lb:
                return False
        return True
    except (oracle.OracleError, AssertionError):
        return False


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "clean.c"
    path.write_text(src)
    so = tmp_path / "libclean.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(path), "-lm"])
    with oracle.use_library(str(so)):
        assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    so = _build_mutant(tmp_path, name)
    with oracle.use_library(so):
        assert not _pins_pass(), f"planted mistake {name} went unnoticed"
