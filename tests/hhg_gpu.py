"""Helpers for the GPU tests: set up a libhhgs context and move fields between the library
layout (entries, component-major) and unique-node order, all through the C ABI."""

import numpy as np

from oracle import fem, mesh, operators as op, solvers as S
from paper_1908_08666_gb300 import binding as B


def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        import pytest

        pytest.skip("no CUDA device")
    return torch


class Ctx:
    def __init__(self, xyz, tets, level, problem=None, dirichlet_face_flags=None, coarsest=None):
        self.torch = torch_cuda()
        self.stream = self.torch.cuda.current_stream().cuda_stream
        self.h = B.hhg_create(0, self.stream)
        B.hhg_set_macro_mesh(self.h, xyz, tets, dirichlet_face_flags)
        if coarsest is not None:
            B.hhg_set_coarsest_level(self.h, coarsest)
        B.hhg_refine(self.h, level)
        B.hhg_set_problem(self.h, **(problem or {}))
        self.level = level
        self.E, self.U, self.F = B.hhg_num_nodes(self.h, level)
        self.coords_e = B.hhg_entry_coords(self.h, level)
        self.e2u, self.udir = B.hhg_entry_to_unique(self.h, level)
        first = np.full(self.U, -1, dtype=np.int64)
        first[self.e2u[::-1]] = np.arange(self.E)[::-1]
        self.coords_u = self.coords_e[first]

    def maps(self, level):
        """(coords_u, e2u, udir, E, U) of any level."""
        E, U, _ = B.hhg_num_nodes(self.h, level)
        ce = B.hhg_entry_coords(self.h, level)
        e2u, udir = B.hhg_entry_to_unique(self.h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        return ce[first], e2u, udir, E, U

    def to_lib_level(self, level, unique_vals, dtype, comps=3):
        t = self.torch
        E, U, _ = B.hhg_num_nodes(self.h, level)
        u = np.asarray(unique_vals, dtype=np.float64).reshape(U, comps).T.copy()
        src = self.dev(u.reshape(-1), dtype)
        dst = t.empty(comps * E, dtype=dtype, device="cuda")
        B.hhg_scatter_unique(self.h, level, B.F64 if dtype == t.float64 else B.F32, comps, src, dst)
        return dst

    def from_lib_level(self, level, field, comps=3):
        t = self.torch
        E, U, _ = B.hhg_num_nodes(self.h, level)
        dst = t.empty(comps * U, dtype=field.dtype, device="cuda")
        B.hhg_gather_unique(self.h, level, B.F64 if field.dtype == t.float64 else B.F32, comps, field, dst)
        t.cuda.synchronize()
        return dst.double().cpu().numpy().reshape(comps, U).T.copy()

    def close(self):
        if self.h:
            B.hhg_destroy(self.h)
            self.h = None

    def dev(self, a, dtype):
        t = self.torch
        return t.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")

    def to_lib(self, unique_vals, dtype, comps):
        """(U, comps) or (U,) host array in unique order -> device field in library layout."""
        t = self.torch
        u = np.asarray(unique_vals, dtype=np.float64).reshape(self.U, comps).T.copy()  # comp-major
        src = self.dev(u.reshape(-1), dtype)
        dst = t.empty(comps * self.E, dtype=dtype, device="cuda")
        B.hhg_scatter_unique(self.h, self.level, B.F64 if dtype == t.float64 else B.F32, comps, src, dst)
        return dst

    def from_lib(self, field, comps):
        t = self.torch
        dst = t.empty(comps * self.U, dtype=field.dtype, device="cuda")
        B.hhg_gather_unique(self.h, self.level, B.F64 if field.dtype == t.float64 else B.F32, comps, field, dst)
        t.cuda.synchronize()
        return dst.double().cpu().numpy().reshape(comps, self.U).T.copy()

    def set_k(self, k_unique, dtype=None):
        t = self.torch
        kd = self.to_lib(k_unique, t.float64, 1)
        B.hhg_set_coefficient(self.h, kd, B.F64)
        t.cuda.synchronize()


NU = 0.3


def kfun_smooth(c):
    return 1.0 + 0.5 * np.sin(3.0 * c[:, 0]) * np.cos(2.0 * c[:, 1]) + 0.3 * c[:, 2]


def oracle_hier(builder, levels, kfun):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    ce, cd = fem.elasticity_coefficients(NU)

    def A_of(lv):
        K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
        return op.with_dirichlet_rows(op.scaled_operator(lv, K, kfun(lv.coords)), lv.dirichlet)

    return S.Hierarchy(mm, levels, A_of)


class Pair:
    """GPU context and oracle hierarchy on the same mesh, with node permutations."""

    def __init__(self, builder, level, kfun=kfun_smooth, coarsest=2):
        self.xyz, self.tets = builder()
        self.level = level
        self.H = oracle_hier(builder, list(range(coarsest, level + 1)), kfun)
        self.ctx = Ctx(self.xyz, self.tets, level, dict(nu=NU), coarsest=coarsest)
        self.ctx.set_k(kfun(self.ctx.coords_u))
        self.perm, self.dirs = {}, {}
        for l in range(coarsest, level + 1):
            cu, _, udir, _, _ = self.ctx.maps(l)
            self.perm[l] = mesh.match_nodes(self.H.lv[l].coords, cu)
            self.dirs[l] = udir

    def to_lib(self, l, x_or, dtype):
        u = np.empty_like(x_or)
        u[self.perm[l]] = x_or
        return self.ctx.to_lib_level(l, u, dtype)

    def from_lib(self, l, field):
        return self.ctx.from_lib_level(l, field)[self.perm[l]]

    def close(self):
        self.ctx.close()
