"""Worker side of the sampled full-size parity tests: rows of the 6-macro cube operator on
the benchmark workload (lognormal E seed 2, x ~ U[-1, 1] seed 3) by the single-row oracle,
evaluated in spawned processes (the test process holds a CUDA context)."""

import hhg_inputs as hi
from oracle import fem, mesh, rows

_W = {}


def init(level):
    xyz, tets = hi.kuhn_cube(1)
    _W.update(level=level, mm=mesh.MacroMesh.build(xyz, tets), gk=hi.lognormal_grid(1 << level, seed=2),
              gx=hi.uniform_grid(1 << level, seed=3), c=fem.elasticity_coefficients(0.3))


def kf(c):
    return hi.sample_grid(_W["gk"][..., None], c)[:, 0]


def xf(c):
    return hi.sample_grid(_W["gx"], c)


def job(items):
    """[(macro, (i, j, k)), ...] -> [(y (3,), term scale (3,)), ...]"""
    ce, cd = _W["c"]
    out = []
    for m, ijk in items:
        y, _, sc = rows.row(_W["mm"], _W["level"], m, ijk, kf, xf, ce, cd, want_scale=True)
        out.append((y, sc))
    return out
