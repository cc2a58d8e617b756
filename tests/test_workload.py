"""The shared seeded input generator: shapes, determinism, subsets, model facts."""
import numpy as np

from paper_2606_05687_b300 import workload as W


def test_shapes_and_dtypes():
    b = W.generate(W.rl_scale_walking(B=5))
    assert b.A.shape == (5, 20, 13, 13) and b.Bm.shape == (5, 20, 13, 24)
    assert b.A.dtype == np.float32 and b.mask.dtype == np.uint32
    s = W.generate(W.small_centroidal(B=3))
    assert s.Bm.shape == (3, 10, 13, 12) and s.mu.shape == (3, 10, 2)


def test_determinism_and_subsets():
    spec = W.rl_scale_walking(B=16)
    a = W.generate(spec)
    b = W.generate(spec)
    sub = W.generate(spec, instances=[3, 11])
    for name in ("A", "Bm", "Q", "R", "ry", "xi0", "mu", "mask"):
        assert np.array_equal(getattr(a, name), getattr(b, name))
        assert np.array_equal(getattr(a, name)[[3, 11]], getattr(sub, name))


def test_model_structure():
    b = W.generate(W.rl_scale_walking(B=4))
    # gravity state is constant: unit row in A, zero row in B
    assert np.all(b.A[..., 12, :12] == 0) and np.all(b.A[..., 12, 12] == 1)
    assert np.all(b.Bm[..., 12, :] == 0)
    # linear-velocity rows of B are dt/m on each force component
    assert np.allclose(b.Bm[..., 6, 0], 0.02 / W.MASS)
    # walking gait: all points of one foot share a stance bit
    st = b.stance()
    assert np.array_equal(st[..., 0:4].min(-1), st[..., 0:4].max(-1))
    assert 0.3 < st.mean() < 0.9


def test_receding_step_shifts_stages():
    b = W.generate(W.rl_scale_walking(B=4, N=6, seed=1002))
    xi0 = np.arange(4 * b.nx, dtype=np.float32).reshape(4, b.nx)
    up = np.ones((4, b.nu), np.float32)
    n = b.receding(xi0, up)
    assert n.B == b.B and n.N == b.N
    for name in ("A", "Bm", "e", "Q", "R", "ry", "ru", "mu", "fmax", "mask"):
        old, new = getattr(b, name), getattr(n, name)
        assert np.array_equal(new[:, :-1], old[:, 1:]), name
        assert np.array_equal(new[:, -1], old[:, -1]), name
    assert np.array_equal(n.xi0, xi0) and np.array_equal(n.u_prev, up)
    assert np.array_equal(n.horizon, b.horizon)


def _cd9_step(xi, f, tau, p, dt):
    """One step of the discrete centroidal dynamics of Sec. II-A, as printed:
    c+ = c + dt l/m,  l+ = l + dt (m g + sum f),  k+ = k + dt sum ((p - c) x f + tau)."""
    c, l, k = xi[0:3], xi[3:6], xi[6:9]
    g = np.array([0.0, 0.0, -W.GRAVITY])
    cn = c + dt * l / W.MASS
    ln = l + dt * (W.MASS * g + f.sum(0))
    kn = k + dt * (np.cross(p - c, f).sum(0) + tau.sum(0))
    return np.concatenate([cn, ln, kn])


def test_cd9_linearisation_against_the_centroidal_dynamics():
    # at c = cbar the linear model equals the nonlinear step for any l, k,
    # forces; elsewhere it exceeds it by exactly dt (c - cbar) x sum(f - fbar)
    rng = np.random.default_rng(11)
    for spec in (W.centroidal9_walking(B=3, N=6), W.centroidal9_small(B=3, N=6)):
        b = W.generate(spec)
        cd, nc = spec.contact_dim, spec.n_contacts
        A, Bm, e = b.A.astype(np.float64), b.Bm.astype(np.float64), b.e.astype(np.float64)
        for i in range(3):
            for k in range(6):
                cbar = b.nominal["cbar"][i, k]
                p = cbar + b.nominal["lever"][i, k]                      # [nc,3]
                st = b.stance()[i, k]
                fbar = np.zeros((nc, 3))
                if st.any():
                    fbar[st, 2] = W.MASS * W.GRAVITY / st.sum()
                for dc_scale in (0.0, 0.05):
                    xi = np.concatenate([cbar + dc_scale * rng.normal(size=3), rng.normal(size=6)])
                    u = rng.normal(size=(nc, cd)) * 20.0
                    u[~st] = 0.0
                    f, tau = u[:, 0:3], (u[:, 3:6] if cd == 6 else np.zeros((nc, 3)))
                    lin = A[i, k] @ xi + Bm[i, k] @ u.reshape(-1) + e[i, k]
                    nonlin = _cd9_step(xi, f[st], tau[st], p[st], spec.dt)
                    want = spec.dt * np.cross(xi[0:3] - cbar, (f - fbar)[st].sum(0)) if st.any() else 0.0
                    got = lin.copy()
                    got[6:9] -= want
                    assert np.allclose(got, nonlin, rtol=0, atol=1e-4 * (1 + np.abs(nonlin).max())), (spec.contact_dim, i, k)


def test_per_instance_horizons_leave_other_draws_unchanged():
    a = W.generate(W.rl_scale_walking(B=64))
    b = W.generate(W.rl_scale_walking(B=64, horizon_min=5))
    assert np.all(a.horizon == 20) and b.horizon.min() >= 5 and b.horizon.max() <= 20 and len(set(b.horizon)) > 8
    for k in ("A", "Bm", "Q", "R", "ry", "xi0", "mu", "mask", "e"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert np.array_equal(W.generate(W.rl_scale_walking(B=64, horizon_min=5), instances=[9, 33]).horizon, b.horizon[[9, 33]])
    parts = W.uneven_mixed(B=100, N=32)
    assert [p.B for p in parts] == [50, 50] and {p.contact_dim for p in parts} == {3, 6}
