"""lbm_reduce_fields_noalloc against lbm_diagnostics.

The allocation-free reduction serves callers that may not call cudaMalloc (a
framework that owns all device memory through its own pool, or a loop that
cannot take the device synchronisation of an allocation). It reduces fields the
caller already holds in device memory; here those fields come from
lbm_get_fields_device into a buffer this test owns, and the 14 results must
equal the context's own diagnostics (lbm_diagnostics) on two calls in a row per
grid, over a sequence of grids: a whole number of 8192-cell blocks (256 x 384),
a ragged one whose last block is partial (250 x 383), then a smaller grid of
one partial block (62 x 97), so that later calls find the shared scratch array
holding more blocks of an earlier call's sums than they launch themselves.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MASK = 1 | 2 | 4 | 16 | 64      # phi, ux, uy, rho, P


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def _expected(d):
    return np.array([d["sum_phi"], d["sum_rho"], d["kinetic_energy"], d["max_u"],
                     d["centroid_A_x"] * d["mass_A"], d["centroid_A_y"] * d["mass_A"],
                     d["centroid_B_x"] * d["mass_B"], d["centroid_B_y"] * d["mass_B"],
                     d["P_bulk_A"] * d["n_bulk_A"], d["n_bulk_A"],
                     d["P_bulk_B"] * d["n_bulk_B"], d["n_bulk_B"], float(d["nonfinite"]),
                     d["mass_B"]])


def _order_bounds(f, eps_r):
    """(2 (n - 1) 2^-53 + 8 eps_r) sum |x_i| for each summed quantity, from the fields."""
    phi, ux, uy, rho, P = f
    ny, nx = phi.shape
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    A, B = phi > 1 - 1e-3, phi < 1e-3
    terms = {0: phi, 1: rho, 2: 0.5 * rho * (ux * ux + uy * uy), 4: phi * x, 5: phi * y,
             6: (1 - phi) * x, 7: (1 - phi) * y, 8: P[A], 10: P[B], 13: 1 - phi}
    return {q: (2 * max(t.size - 1, 1) * 2.0 ** -53 + 8 * eps_r) * np.abs(t).sum()
            for q, t in terms.items()}


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_noalloc_reduction_matches_diagnostics_twice(L, form):
    import torch
    from paper_1902_08933_gb300 import workloads as wl
    stream = torch.cuda.Stream()
    out = torch.empty(14, dtype=torch.float64, device="cuda")
    for nx, ny, R, cy in ((256, 384, 40, 120), (250, 383, 40, 120), (62, 97, 12, 30)):
        cfg = wl.rising_bubble(nx=nx, ny=ny, R=R, cy=cy, W=4.0, Re=20.0)
        fields = torch.empty(5 * nx * ny, dtype=torch.float64, device="cuda")
        with L.Simulation(cfg, form, stream=stream.cuda_stream, phi0=[wl.initial_phi(cfg)]) as sim:
            for call in range(2):
                sim.step(25)
                L.lbm_get_fields_device(sim.ctx, 0, MASK, fields.data_ptr())
                out.fill_(float("nan"))
                st = L.lbm_reduce_fields_noalloc(fields.data_ptr(), nx, ny, stream.cuda_stream,
                                                 out.data_ptr())
                assert st == L.LBM_OK
                stream.synchronize()
                got = out.cpu().numpy()
                exp = _expected(sim.diagnostics())
                # Sums: per-cell terms added in another order. Recursive summation
                # of n terms errs by at most (n - 1) 2^-53 sum|x_i|, so two orders
                # differ by at most twice that. The per-cell values come from the
                # same formulas compiled into two kernels, which may round them a
                # few ulps of the arithmetic type apart (FMA contraction), hence
                # 8 eps_R sum|x_i|; plus a few ulps of the centroid * mass
                # reconstruction.
                eps_r = 2.0 ** -53 if form == "f64" else 2.0 ** -24
                bound = _order_bounds(fields.cpu().numpy().reshape(5, ny, nx), eps_r)
                for q in (0, 1, 2, 4, 5, 6, 7, 8, 10, 13):
                    tol = bound[q] + 4 * 2.0 ** -53 * abs(exp[q])
                    assert abs(got[q] - exp[q]) <= tol, ((nx, ny), call, q, got[q], exp[q], tol)
                for q in (3, 9, 11, 12):         # max and counts: exact
                    assert got[q] == exp[q], ((nx, ny), call, q, got[q], exp[q])


def test_noalloc_rejects_oversized_and_null(L):
    import torch
    buf = torch.empty(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert L.lbm_reduce_fields_noalloc(p, 4097, 4096, None, p) == L.LBM_EINVAL   # > 16,777,216 cells
    assert L.lbm_reduce_fields_noalloc(0, 4, 4, None, p) == L.LBM_EINVAL
    assert L.lbm_reduce_fields_noalloc(p, 4, 4, None, 0) == L.LBM_EINVAL
    assert L.lbm_reduce_fields_noalloc(p, 0, 4, None, p) == L.LBM_EINVAL
