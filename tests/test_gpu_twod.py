"""2D variant of the stencil scaling (Sec. 2.3) on the GPU against the 2D oracle."""

import numpy as np
import pytest

from oracle import twod as T
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import torch_cuda

pytestmark = pytest.mark.gpu

NU = 0.3
FP32_C = 64 * 2.0**-24
TRIS = {"unit": [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], "skewed": [[0.2, 0.1], [1.3, 0.4], [0.5, 1.7]]}


@pytest.mark.parametrize("name", list(TRIS))
@pytest.mark.parametrize("level", [3, 5])
@pytest.mark.parametrize("variant", ["physical", "unphysical", "nodal"])
def test_apply_2d_parity(name, level, variant):
    torch = torch_cuda()
    tri = np.array(TRIS[name])
    lat = T.Lattice2D(tri, level)
    ce, cd = 1.0 / (1.0 + NU), NU / ((1.0 + NU) * (1.0 - 2.0 * NU))
    K = T.element_stiffness(lat.coords[lat.elems], ce, cd)
    c = lat.coords
    k = 1.0 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1]) + 0.2 * c[:, 0]
    A = T.operator(lat, K, k, variant)
    x = np.random.default_rng(level).uniform(-1, 1, (lat.N, 2))
    want = T.apply(A, x)
    # FP32 row bound as for 3D: 64 * 2^-24 * sum_j |A_ij| |x_j - x_i| (the difference form the
    # kernel evaluates; row r = 2 i + m, column q = 2 j + l, x_i taken in the column's component)
    rows, cols = np.nonzero(A)
    xf = x.reshape(-1)
    scale = np.zeros(2 * lat.N)
    np.add.at(scale, rows, np.abs(A[rows, cols]) * np.abs(xf[cols] - xf[(rows // 2) * 2 + cols % 2]))
    scale = scale.reshape(-1, 2)
    h = B.hhg_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        var = {"physical": B.PHYSICAL, "unphysical": B.UNPHYSICAL, "nodal": B.NODAL}[variant]
        for dt, tdt in ((B.F64, torch.float64), (B.F32, torch.float32)):
            kd = torch.as_tensor(k, dtype=tdt, device="cuda")
            xd = torch.as_tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=tdt, device="cuda")
            yd = torch.empty_like(xd)
            B.hhg_apply_2d(h, tri, level, NU, var, dt, kd, xd, yd)
            got = yd.double().cpu().numpy().reshape(2, lat.N).T
            if dt == B.F64:
                assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
            else:
                inner = ~lat.boundary
                assert np.all(np.abs(got - want)[inner] <= FP32_C * scale[inner] + 1e-30)
                assert np.abs(got - want)[~inner].max() <= 2**-24 * np.abs(x).max()
        with pytest.raises(B.HhgError):
            B.hhg_apply_2d(h, [[0, 0], [1, 1], [2, 2]], level, NU, var, B.F64, kd, xd, yd)  # degenerate
    finally:
        B.hhg_destroy(h)
