"""Pins of the oracle's building blocks against textbook identities, library
routines and closed forms (no GPU)."""
import numpy as np
import pytest
import torch

from paper_0809_4958_gb300 import inputs


def test_d3q19_lattice_isotropy(orc):
    # textbook D3Q19 (Sec. 3 names the model): weights 1/3, 1/18, 1/36;
    # moments of the weights up to fourth order are those of an isotropic
    # Gaussian with cs^2 = 1/3.
    c, w = orc.lattice()
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    cs2 = 1.0 / 3.0
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, cs2 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # |c|^2 = 0, 1, 2 for the three shells and opposite pairs sit side by side
    n2 = (c * c).sum(1)
    assert n2[0] == 0 and np.all(n2[1:7] == 1) and np.all(n2[7:] == 2)
    for i in range(1, 19, 2):
        assert np.all(c[i] == -c[i + 1])
    assert len({tuple(v) for v in c}) == 19


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.02, (0.05, -0.03, 0.01)), (0.97, (-0.1, 0.2, 0.07))])
def test_equilibrium_moments(orc, rho, u):
    # sum feq = rho, sum c feq = rho u, sum c c feq = rho (cs^2 I + u u)
    c, _ = orc.lattice()
    feq = orc.equilibrium(rho, u)
    u = np.asarray(u)
    assert abs(feq.sum() - rho) < 1e-15
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", feq, c, c)
    assert np.allclose(P, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-15)


def test_round_f16_matches_numpy(orc):
    # binary16 round-to-nearest-even from double: numpy's float64->float16 cast
    rng = np.random.default_rng(0)
    xs = np.concatenate([
        rng.normal(0, 1e-2, 2000), rng.normal(0, 1e-5, 500), rng.normal(0, 1e-7, 200),  # subnormals
        rng.normal(0, 3e4, 200),
        # exact ties between binary16 neighbours
        (np.arange(1, 200) + 0.5) * 2.0 ** -10, (np.arange(1, 50) + 0.5) * 2.0 ** -24,
        [0.0, 65504.0, 65519.0, 65520.0, -65521.0],
    ])
    for x in xs:
        ref = float(np.float64(x).astype(np.float16))
        got = orc.round_f16(float(x))
        assert got == ref or (np.isinf(ref) and np.isinf(got) and np.sign(ref) == np.sign(got)), (x, got, ref)


def test_round_bf16_matches_torch(orc):
    # bfloat16 round-to-nearest-even: torch's float32 -> bfloat16 cast, on
    # float32 inputs (so the cast is a single rounding)
    rng = np.random.default_rng(1)
    xs32 = np.concatenate([rng.normal(0, 1e-2, 3000), rng.normal(0, 1e-30, 200)]).astype(np.float32)
    ties = ((np.arange(1, 256, dtype=np.float32) * 2 + 1) * np.float32(2.0 ** -16)).astype(np.float32)  # midpoints
    xs32 = np.concatenate([xs32, ties])
    ref = torch.from_numpy(xs32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.round_bf16(float(v)) for v in xs32])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ctr,key,expect", [
    # known-answer vectors published with the Philox generators (Random123)
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox4x32_known_answers(orc, ctr, key, expect):
    assert [int(v) for v in orc.philox4x32_10(ctr, key)] == expect


@pytest.mark.parametrize("eps", [0.0, 1.0])
def test_chain_force_is_minus_gradient(orc, eps):
    # FENE bonds plus WCA pair repulsion (Kremer-Grest): force = -grad U
    # a folded chain: beads 0 and 3 are a non-bonded contact inside the WCA range
    pos = 5.0 + np.array([[0, 0, 0], [0.97, 0, 0], [0.97, 0.97, 0], [0.05, 1.0, 0.1], [-0.9, 1.3, 0.2],
                          [-1.5, 2.1, 0.5], [-1.2, 3.0, 0.9], [-0.6, 3.7, 1.2]])
    k, R0, sig = 30.0, 1.5, 1.0
    st, F = orc.chain_forces(pos, k, R0, eps, sig)
    assert st == 0

    def U(p):
        r = np.diff(p, axis=0)
        r2 = (r * r).sum(1)
        u = float(np.sum(-0.5 * k * R0 ** 2 * np.log(1 - r2 / R0 ** 2)))
        for i in range(len(p)):
            for j in range(i + 1, len(p)):
                d2 = float(((p[j] - p[i]) ** 2).sum())
                if d2 < 2 ** (1 / 3) * sig ** 2:
                    s6 = (sig ** 2 / d2) ** 3
                    u += 4 * eps * (s6 * s6 - s6) + eps
        return u

    h = 1e-6
    for b in range(pos.shape[0]):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[b, a] += h
            pm[b, a] -= h
            assert abs(-(U(pp) - U(pm)) / (2 * h) - F[b, a]) < 1e-6 * max(1.0, abs(F[b, a]))
    assert np.allclose(F.sum(0), 0.0, atol=1e-12)  # Newton's third law
    assert float(((pos[3] - pos[0]) ** 2).sum()) < 2 ** (1 / 3)  # the contact is inside the WCA range
    bad = pos.copy()
    bad[5] = bad[4] + [1.6, 0, 0]
    assert orc.chain_forces(bad, k, R0, eps, sig)[0] == orc.ERR_FENE


def _face_series(E, J, fn):
    """samples[j][f][c][q][p] = fn(j, f, c, q, p) evaluated over arrays."""
    j, f, c, q, p = np.meshgrid(np.arange(J), np.arange(6), np.arange(3), np.arange(E), np.arange(E), indexing="ij")
    return np.ascontiguousarray(fn(j, f, c, q, p).astype(np.float64))


def test_time_interpolation_linear_exact_on_linear_data(orc):
    E, K, J = 8, 5, 6
    S = _face_series(E, J, lambda j, f, c, q, p: 0.01 * (1 + f + 2 * c) + 1e-3 * (q - p) + 2e-3 * j * (c + 1))
    box = orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_LINEAR)
    for n in range(0, (J - 1) * K):
        t = n + 1
        for (f, p, q) in [(0, 1, 2), (3, 7, 0), (5, 4, 4)]:
            st, u = orc.face_velocity(box, S, n, f, p, q)
            assert st == 0
            exact = [0.01 * (1 + f + 2 * c) + 1e-3 * (q - p) + 2e-3 * (t / K) * (c + 1) for c in range(3)]
            assert np.allclose(u, exact, atol=1e-16, rtol=1e-14)
    assert orc.face_velocity(box, S, (J - 1) * K, 0, 0, 0)[0] == orc.ERR_SAMPLES


def test_time_interpolation_hermite_exact_on_quadratics(orc):
    # Catmull-Rom tangents are exact derivatives of a quadratic, so the cubic
    # Hermite reproduces it on every interval after the first
    E, K, J = 8, 4, 7
    a, b, cq = 0.02, -3e-3, 4e-4
    S = _face_series(E, J, lambda j, f, c, q, p: (a + b * j + cq * j * j) * (1 + 0.1 * c) + 1e-4 * (p + f))
    box = orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_HERMITE)
    for n in range(K, (J - 2) * K):
        t = (n + 1) / K
        st, u = orc.face_velocity(box, S, n, 2, 3, 5)
        assert st == 0
        exact = [(a + b * t + cq * t * t) * (1 + 0.1 * c) + 1e-4 * (3 + 2) for c in range(3)]
        assert np.allclose(u, exact, atol=1e-16, rtol=1e-13)
    # at the sample times themselves the Hermite value is the sample
    for j in range(1, J - 2):
        st, u = orc.face_velocity(box, S, j * K - 1, 4, 1, 6)
        assert np.allclose(u, S[j, 4, :, 6, 1], atol=1e-17, rtol=1e-14)
    # the learned residual is added on top of the Hermite value
    box_m = orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_MLP)
    R = np.zeros((6, 3, K, E, E))
    R[1, 2, 2, 3, 0] = 0.125
    n = 2 * K + 2  # s = 3 -> residual slot 2
    u_h = orc.face_velocity(box, S, n, 1, 0, 3)[1]
    u_m = orc.face_velocity(box_m, S, n, 1, 0, 3, resid=R)[1]
    assert np.allclose(u_m - u_h, [0, 0, 0.125], atol=1e-16)


def test_generator_closed_forms(orc):
    E = 16
    xc = 0.5 * (E - 1)
    # at the box centre at t = 0 with zero phases the field is the sum of the amplitudes
    rng = np.random.default_rng(2)
    kv = rng.normal(size=(5, 3))
    am = rng.normal(size=(5, 3))
    m = inputs.Modes(kvec=kv, amp=am, omega=rng.uniform(0, 1, 5), phi=np.zeros(5), E=E, u_max=0.0)
    assert np.allclose(orc.field(m, E, [[xc, xc, xc]], 0.0)[0], am.sum(0), atol=1e-14)
    # a quarter-period phase shift cancels it
    m2 = inputs.Modes(kvec=kv, amp=am, omega=np.zeros(5), phi=np.full(5, np.pi / 2), E=E, u_max=0.0)
    assert np.allclose(orc.field(m2, E, [[xc, xc, xc]], 0.0)[0], 0.0, atol=1e-14)
    # one mode: periodic in time with 2 pi / omega and in space along kvec
    one = inputs.single_mode(E, [0.3, -0.2, 0.1], [0.0, 0.01, 0.02], omega=0.05, phi=0.4)
    x = np.array([[3.0, 7.5, 1.25]])
    u0 = orc.field(one, E, x, 11.0)
    assert np.allclose(orc.field(one, E, x, 11.0 + 2 * np.pi / 0.05), u0, atol=1e-15)
    kk = np.array([0.3, -0.2, 0.1])
    assert np.allclose(orc.field(one, E, x + 2 * np.pi * kk / (kk @ kk), 11.0), u0, atol=1e-15)
    # superposition: the field of a table is the sum of the fields of its halves
    mt = inputs.mode_table(5, 64, 1, 8, E)
    h1 = inputs.Modes(mt.kvec[:30].copy(), mt.amp[:30].copy(), mt.omega[:30].copy(), mt.phi[:30].copy(), E, 0)
    h2 = inputs.Modes(mt.kvec[30:].copy(), mt.amp[30:].copy(), mt.omega[30:].copy(), mt.phi[30:].copy(), E, 0)
    pts = rng.uniform(0, E - 1, (20, 3))
    assert np.allclose(orc.field(mt, E, pts, 7.0), orc.field(h1, E, pts, 7.0) + orc.field(h2, E, pts, 7.0), atol=1e-15)


def test_generator_divergence_free_and_normalised(orc):
    E = 32
    mt = inputs.mode_table(0, 256, 1, 16, E)
    # divergence by central differences at random points: zero to O(h^2)
    rng = np.random.default_rng(3)
    pts = rng.uniform(2, E - 3, (50, 3))
    h = 1e-3
    div = np.zeros(50)
    grad_scale = 0.0
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        d = (orc.field(mt, E, pts + e, 5.0) - orc.field(mt, E, pts - e, 5.0)) / (2 * h)
        div += d[:, a]
        grad_scale = max(grad_scale, np.abs(d).max())
    assert np.abs(div).max() < 1e-6 * grad_scale
    # max |u(x, 0)| over all sites: exactly u_max for E < 64 (the sample lattice is every site)
    u0 = orc.volume_field(mt, E, 0.0)
    assert abs(np.sqrt((u0 ** 2).sum(0)).max() - 0.05) < 1e-12
    # face samples are the field at the face sites at t = j K
    K = 3
    S = orc.face_samples(mt, E, K, 2, 2)
    for (j, f, p, q) in [(0, 0, 5, 9), (1, 1, 0, 31), (0, 2, 7, 3), (1, 3, 30, 2), (0, 4, 11, 12), (1, 5, 1, 0)]:
        axis, val = f // 2, (0 if f % 2 == 0 else E - 1)
        P = {0: [val, p, q], 1: [p, val, q], 2: [p, q, val]}[axis]
        assert np.allclose(S[j, f, :, q, p], orc.field(mt, E, [P], (2 + j) * K)[0], atol=1e-16)
    # volume field layout [c][z][y][x]
    assert np.allclose(u0[:, 4, 9, 2], orc.field(mt, E, [[2, 9, 4]], 0.0)[0], atol=1e-16)
