"""Oracle pins for the spatial zoom (Sec. 3): the boundary samples and the
initial field live on a coarse grid with spacing z lattice sites; the boundary
is bilinear within each face between the time-interpolated coarse values, the
initial field trilinear.  Both are exact on fields linear in space."""
import numpy as np
import pytest

import oracle as orc

G = np.array([[1e-3, -2e-3, 5e-4], [3e-4, 1e-3, -1e-3], [-7e-4, 2e-4, 6e-4]])
A0 = np.array([0.01, -0.02, 0.005])
DT = np.array([2e-5, -1e-5, 3e-5])


def linear_field(X, Y, Z, t):
    """u_c = A0_c + G_c . (x, y, z) + DT_c t, on arrays of coordinates."""
    return np.stack([A0[c] + G[c, 0] * X + G[c, 1] * Y + G[c, 2] * Z + DT[c] * t for c in range(3)])


def coarse_faces(E, z, K, nsamp):
    """Face samples [nsamp][6][3][Ec][Ec] of the linear field at the coarse points."""
    Ec = orc.coarse_points(E, z)
    P = np.arange(Ec) * z
    out = np.zeros((nsamp, 6, 3, Ec, Ec))
    for j in range(nsamp):
        t = j * K
        for f in range(6):
            fixed = 0 if f % 2 == 0 else E - 1
            Qg, Pg = np.meshgrid(P, P, indexing="ij")  # [q][p]
            F = np.full_like(Pg, fixed, dtype=np.float64)
            xyz = [(F, Pg, Qg), (Pg, F, Qg), (Pg, Qg, F)][f // 2]
            out[j, f] = linear_field(*xyz, t)
    return out


@pytest.mark.parametrize("E,z", [(31, 2), (31, 3), (31, 5), (16, 6), (24, 5)])
@pytest.mark.parametrize("interp", [orc.TIME_LINEAR, orc.TIME_HERMITE])
def test_bilinear_boundary_exact_on_linear_fields(E, z, interp):
    # (16, 6) and (24, 5): the last coarse cell reaches past the box
    K = 4
    box = orc.BoxParams(E=E, tau=0.8, K=K, time_interp=interp, zoom=z)
    S = coarse_faces(E, z, K, 6)
    for n in (0, 3, 6):
        t = n + 1
        for f in range(6):
            for p, q in [(0, 0), (1, 2), (E - 1, 7), (13, E - 1), (E - 2, E - 2)]:
                st, u = orc.face_velocity(box, S, n, f, p, q)
                assert st == 0
                fixed = 0 if f % 2 == 0 else E - 1
                xyz = [(fixed, p, q), (p, fixed, q), (p, q, fixed)][f // 2]
                assert np.allclose(u, linear_field(*xyz, t), rtol=0, atol=1e-15), (n, f, p, q)


def test_bilinear_boundary_between_coarse_points():
    # a field that is not linear: at a coarse point the sample itself, half way
    # between two coarse points the mean of the two
    E, z = 13, 3
    box = orc.BoxParams(E=E, tau=0.8, K=1, zoom=z)
    Ec = orc.coarse_points(E, z)
    rng = np.random.default_rng(0)
    S = rng.normal(0, 0.01, (3, 6, 3, Ec, Ec))
    for f in (0, 3, 5):
        st, u = orc.face_velocity(box, S, 0, f, 2 * z, z)  # t = 1: sample 1 exactly
        assert st == 0 and np.array_equal(u, S[1, f, :, 1, 2])
        st, u = orc.face_velocity(box, S, 0, f, 0, 1)  # one third of the way from (0,0) to (0,1) in q
        assert np.allclose(u, (2 * S[1, f, :, 0, 0] + S[1, f, :, 1, 0]) / 3, rtol=0, atol=1e-17)


@pytest.mark.parametrize("E,z", [(17, 2), (17, 4), (16, 3), (16, 6)])
def test_trilinear_initial_field_exact_on_linear_fields(E, z):
    box = orc.BoxParams(E=E, tau=0.8, zoom=z)
    Ec = box.coarse_points()
    C = np.arange(Ec) * z
    Zc, Yc, Xc = np.meshgrid(C, C, C, indexing="ij")
    f = orc.init(box, linear_field(Xc, Yc, Zc, 0.0))
    Zs, Ys, Xs = np.meshgrid(np.arange(E), np.arange(E), np.arange(E), indexing="ij")
    fine = orc.init(orc.BoxParams(E=E, tau=0.8), linear_field(Xs, Ys, Zs, 0.0))
    assert np.max(np.abs(f - fine)) <= 1e-15


def test_zoomed_run_equals_every_site_run_on_a_linear_field():
    # the boundary and the initial field of a field linear in space are the
    # same whether sampled at every site or on the coarse grid, so the runs
    # agree to rounding (the interior flow itself need not stay linear)
    E, z, K, steps = 19, 3, 2, 12
    Zs, Ys, Xs = np.meshgrid(np.arange(E), np.arange(E), np.arange(E), indexing="ij")
    every = orc.Sim(orc.BoxParams(E=E, tau=0.9, K=K), linear_field(Xs, Ys, Zs, 0.0), coarse_faces(E, 1, K, steps // K + 3))
    box = orc.BoxParams(E=E, tau=0.9, K=K, zoom=z)
    C = np.arange(box.coarse_points()) * z
    Zc, Yc, Xc = np.meshgrid(C, C, C, indexing="ij")
    zoomed = orc.Sim(box, linear_field(Xc, Yc, Zc, 0.0), coarse_faces(E, z, K, steps // K + 3))
    assert every.run(steps) == 0 and zoomed.run(steps) == 0
    assert np.max(np.abs(every.f - zoomed.f)) <= 1e-15


def test_generator_on_the_coarse_grid():
    from paper_0809_4958_gb300 import inputs
    E, z = 25, 4
    modes = inputs.mode_table(2, 16, 1.0, 6.0, E)
    full = orc.face_samples(modes, E, 3, 1, 2)
    coarse = orc.face_samples(modes, E, 3, 1, 2, zoom=z)
    assert np.array_equal(coarse, full[:, :, :, ::z, ::z])
    vfull = orc.volume_field(modes, E, 0.5)
    vcoarse = orc.volume_field(modes, E, 0.5, zoom=z)
    assert np.array_equal(vcoarse, vfull[:, ::z, ::z, ::z])
