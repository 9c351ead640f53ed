"""Pins of the oracle's set-up relaxation (paper Sec. 3, Eq. relax).

The first vector set comes from nu sweeps e <- (1 - omega A_l) e on random
starts, with omega = 1 / lambda~max and lambda~max the Rayleigh quotient of a
power iteration.  Everything here is fixed by the spectral decomposition of
the level's Hermitian operator, formed densely in the test (A = D^dagger D
from the explicit Dirac matrix at level 0; the dense P^dagger A P, formed from
the dense prolongator, at level 1), never by re-running the oracle's loops:

* after k power iterations from v0 = sum_i c_i q_i the Rayleigh quotient is
  sum |c_i|^2 lam_i^(2k-1) / sum |c_i|^2 lam_i^(2k-2), and it lies below
  lambda_max;
* the relaxed vectors equal Q diag((1 - omega lam_i)^nu) Q^dagger e0 with
  omega from that closed form;
* the quotient never exceeds lambda_max, so omega >= 1/lambda_max, and with
  omega < 2/lambda_max every factor |1 - omega lam| is below 1: each sweep
  shrinks the vector in the 2-norm and in the A-norm.

A changed omega (e.g. 0.3 / lambda) or a changed sweep count fails the second
pin; a changed power-iteration count fails the first.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg
from oracle import wilson as w


def _noise_slices(shapes, Nv, noise):
    """Per relaxed level: (starts, power start, MR start) in the set-up noise
    layout (Nv starts, then the power-iteration start, then the smoother start)."""
    out, pos = [], 0
    for (lx, lt, n), nv in zip(shapes[:-1], Nv):
        size = lx * lt * n
        starts = noise[pos:pos + nv * size].reshape(nv, lt, lx, n)
        pos += nv * size
        pw = noise[pos:pos + size].reshape(lt, lx, n)
        pos += size
        pos += size
        out.append((starts, pw))
    return out


def _dense_P(lv):
    Ltc, Lxc = lv.Lt // lv.bt, lv.Lx // lv.bx
    nc = Ltc * Lxc * 2 * lv.Nv
    cols = []
    for i in range(nc):
        e = np.zeros(nc, dtype=np.complex128)
        e[i] = 1
        cols.append(mg.prolong(lv.V, lv.bx, lv.bt, e.reshape(Ltc, Lxc, 2 * lv.Nv)).ravel())
    return np.stack(cols, axis=1)


def _build(L, blocks, Nv, m=-0.6, beta=3.0, sweeps=8, power_iters=30):
    Lx, Lt = L
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, beta, 20, 3))
    noise = W.setup_noise(Lx, Lt, blocks, Nv, 11)
    H = mg.setup(U, m, list(blocks), list(Nv), noise, sweeps=sweeps, power_iters=power_iters)
    shapes = W.level_shapes(Lx, Lt, blocks, Nv)
    D = w.dirac_matrix(U, m).toarray()
    A0 = D.conj().T @ D
    dense = [A0]
    for lv in H.levels[:-2]:
        P = _dense_P(lv)
        dense.append(P.conj().T @ dense[-1] @ P)
    return H, dense, _noise_slices(shapes, Nv, noise)


def _rayleigh_closed_form(lam, Q, v0, k):
    c2 = np.abs(Q.conj().T @ v0.ravel()) ** 2
    return float(np.sum(c2 * lam ** (2 * k - 1)) / np.sum(c2 * lam ** (2 * k - 2)))


CASES = [((8, 8), ((2, 2),), (3,)), ((16, 16), ((4, 4), (2, 2)), (3, 4))]


@pytest.mark.parametrize("L,blocks,Nv", CASES)
def test_power_iteration_matches_spectral_closed_form(L, blocks, Nv):
    H, dense, sl = _build(L, blocks, Nv)
    for l, (A, (starts, pw)) in enumerate(zip(dense, sl)):
        lam, Q = np.linalg.eigh(A)
        assert lam[0] > 0
        for k in (1, 2, 30):
            rq = mg.power_lambda_max(H.levels[l].op.apply, pw, k)
            ref = _rayleigh_closed_form(lam, Q, pw, k)
            assert abs(rq - ref) <= 1e-12 * lam[-1], (l, k, rq, ref)
            assert rq <= lam[-1] * (1 + 1e-13)
        # the set-up's omega is the reciprocal of the 30-iteration quotient
        om = 1.0 / _rayleigh_closed_form(lam, Q, pw, 30)
        assert abs(H.levels[l].omega_relax - om) <= 1e-12 * om
        # and 30 iterations bring the quotient close to lambda_max on these operators
        assert _rayleigh_closed_form(lam, Q, pw, 30) >= 0.9 * lam[-1]


@pytest.mark.parametrize("L,blocks,Nv", CASES)
def test_relaxed_vectors_equal_spectral_filter(L, blocks, Nv):
    nu = 8
    H, dense, sl = _build(L, blocks, Nv, sweeps=nu)
    for l, (A, (starts, pw)) in enumerate(zip(dense, sl)):
        lam, Q = np.linalg.eigh(A)
        om = 1.0 / _rayleigh_closed_form(lam, Q, pw, 30)
        filt = (1.0 - om * lam) ** nu
        E = H.levels[l].E
        for k in range(starts.shape[0]):
            ref = Q @ (filt * (Q.conj().T @ starts[k].ravel()))
            err = np.max(np.abs(E[k].ravel() - ref))
            assert err <= 1e-12 * np.max(np.abs(starts[k])), (l, k, err)
        # a different relaxation step or sweep count gives other vectors
        for om_bad, nu_bad in ((0.3 * om, nu), (om, nu - 2), (om, nu + 1)):
            ref = Q @ ((1.0 - om_bad * lam) ** nu_bad * (Q.conj().T @ starts[0].ravel()))
            assert np.max(np.abs(E[0].ravel() - ref)) > 1e-6 * np.max(np.abs(starts[0]))


@pytest.mark.parametrize("L,blocks,Nv", CASES)
def test_relaxation_contracts_every_mode(L, blocks, Nv):
    H, dense, sl = _build(L, blocks, Nv, sweeps=1)
    for l, (A, (starts, pw)) in enumerate(zip(dense, sl)):
        lam = np.linalg.eigvalsh(A)
        om = H.levels[l].omega_relax
        # the quotient never exceeds lambda_max, so omega >= 1/lambda_max; it
        # stays below 2/lambda_max, so |1 - omega lam| < 1 on the whole spectrum
        assert 1 - 1e-13 <= om * lam[-1] < 2
        assert np.max(np.abs(1 - om * lam)) < 1
        for k in range(starts.shape[0]):
            e = starts[k].ravel()
            n2, nA = np.inf, np.inf
            for _ in range(10):
                n2_new = np.linalg.norm(e)
                nA_new = np.sqrt(np.vdot(e, A @ e).real)
                assert n2_new <= n2 * (1 + 1e-13) and nA_new <= nA * (1 + 1e-13)
                n2, nA = n2_new, nA_new
                e = e - om * (A @ e)
        # the first sweep the set-up made is the dense one
        e1 = starts[0].ravel() - om * (A @ starts[0].ravel())
        assert np.max(np.abs(H.levels[l].E[0].ravel() - e1)) <= 1e-13 * np.max(np.abs(e1))
