"""Lifted states, fidelities and observables through the GPU path.

* The q lowest states lifted to the 2^N basis (Eq. (11) applied recursively)
  against the oracle's lifted states: the overlap of the two retained
  subspaces (singular values of psi_or^T psi_gpu), 1 - 1e-9 for the FP64 path
  and 1 - 1e-7 for the mixed paths.
* The ten-site fidelity claim of Sec. III A (two five-site Ising modules,
  h = 0.7, k = 7, Eq. (16) against exact diagonalisation): the GPU's
  fidelities equal the oracle's, and the claim's thresholds hold as read.
* Observables <psi_mu|O|psi_nu> carried through the basis rotations to the
  top block, against the same matrix elements of the oracle's lifted states
  and of the GPU's own lifted states.
"""
import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu
STATE_TOL = {"fp64": 1e-9, "mixed": 1e-7, "mixed_tf32": 1e-7}
OBS_TOL = {"fp64": 1e-9, "mixed": 1e-6, "mixed_tf32": 1e-6}
PAULI = {"X": np.array([[0.0, 1.0], [1.0, 0.0]]), "Z": np.array([[1.0, 0.0], [0.0, -1.0]]),
         "Y": np.array([[0.0, 1.0], [-1.0, 0.0]])}  # Y as the real iY


@pytest.fixture(scope="module", params=["fp64", "mixed", "mixed_tf32"])
def ctx(request):
    torch_cuda()
    c = P.Context(precision=request.param)
    yield c
    c.close()


STATE_CHAINS = [
    I.tfim(12, 1.0, 1.1, 3, 16, 4),
    I.xxz(10, list(np.random.default_rng(51).uniform(0.5, 1.5, 9)), 0.6, 5, 12, 3,
          fields=list(np.random.default_rng(52).uniform(-0.5, 0.5, 10))),
    I.tfim_nnn(14, 1.0, 0.9, 0.2, 4, 16, 4),
    I.tfim(18, 1.0, 0.9, 9, 48, 3),            # wide leaves (exact sub-leaf merges)
    I.tfim(7, 1.0, 0.8, 7, 8, 4),              # the whole chain is one leaf
]


@pytest.mark.parametrize("chain", STATE_CHAINS, ids=lambda c: c.name)
def test_lifted_states_match_oracle(ctx, chain):
    E, _, psi = ctx.solve_chain_states(chain, states=True)
    r = O.solve(chain)
    ref = O.lift_states(r.top)[:, :chain.q]
    np.testing.assert_allclose(E, r.energies, atol=1e-8 * max(1.0, np.abs(r.energies).max()))
    got = psi.T
    np.testing.assert_allclose(got.T @ got, np.eye(chain.q), atol=1e-10)
    sv = np.linalg.svd(ref.T @ got, compute_uv=False)
    assert sv.min() >= 1 - STATE_TOL[ctx.precision], sv


def _fidelity(w, V, psi, mu, tol=1e-9):
    members = np.where(np.abs(w - w[mu]) < tol * max(1.0, abs(w[mu])))[0]
    proj = V[:, members].T @ psi[:, mu]
    return float(proj @ proj)


@pytest.mark.parametrize("Jp", [0.0, 0.25, 0.5, 0.75, 0.85, 1.0])
def test_ten_site_fidelity_claim(ctx, Jp):
    """Sec. III A: k = 7 keeps F > 0.99 for the low-lying states (the three
    lowest over J' in [0, 1], the fourth up to J' = 0.85, as read)."""
    c = I.two_module_tfim("I", Jp, 7)
    _, _, psi = ctx.solve_chain_states(c, states=True)
    w, V = np.linalg.eigh(O.full_chain_hamiltonian(c))
    ref = O.lift_states(O.solve(c).top)
    for mu in range(4):
        f_gpu = _fidelity(w, V, psi.T, mu)
        f_or = _fidelity(w, V, ref, mu)
        assert abs(f_gpu - f_or) <= 10 * STATE_TOL[ctx.precision], (mu, f_gpu, f_or)
        if mu < 3 or Jp <= 0.85:
            assert f_gpu > 0.99, (mu, f_gpu)


OBS_CHAINS = [I.tfim(12, 1.0, 1.3, 3, 16, 4), I.tfim_nnn(10, 1.0, 1.2, 0.2, 5, 12, 3)]


@pytest.mark.parametrize("chain", OBS_CHAINS, ids=lambda c: c.name)
def test_observables_match_lifted_states(ctx, chain):
    """<psi_mu|O|psi_nu> of single-site X, Z and iY carried to the top block:
    diagonals (gauge-invariant for these non-degenerate states) and the
    magnitudes of off-diagonals, against the oracle's lifted states; the whole
    matrices against the GPU's own lifted states (same gauge)."""
    N = chain.n_sites
    obs = [(0, "X"), (N // 2, "X"), (N - 1, "Z"), (1, "Z"), (2, "Y")]
    E, M, psi = ctx.solve_chain_states(chain, observables=obs, states=True)
    ref = O.lift_states(O.solve(chain).top)[:, :chain.q]
    tol = OBS_TOL[ctx.precision]
    for o, (site, p) in enumerate(obs):
        Op = O.site_operator(PAULI[p], site, 0, N)
        want = ref.T @ Op @ ref
        own = psi @ Op @ psi.T
        np.testing.assert_allclose(M[o], own, atol=tol)
        np.testing.assert_allclose(np.diag(M[o]), np.diag(want), atol=tol)
        np.testing.assert_allclose(np.abs(M[o]), np.abs(want), atol=tol)
        if p == "Y":
            np.testing.assert_allclose(M[o], -M[o].T, atol=tol)
        else:
            np.testing.assert_allclose(M[o], M[o].T, atol=tol)


def test_observables_on_a_long_chain(ctx):
    """Carried observables need no lifting: a 64-site chain, where <X_s> of
    the ground state matches the same site's value from the left-right
    mirror-image chain (the chain is reflection-symmetric), and every
    expectation value is in [-1, 1]."""
    c = I.tfim(64, 1.0, 1.3, 4, 16, 2)
    obs = [(s, "X") for s in (0, 5, 31, 32, 58, 63)]
    E, M, _ = ctx.solve_chain_states(c, observables=obs)
    d = np.array([M[o][0, 0] for o in range(len(obs))])
    assert np.all(np.abs(d) <= 1 + 1e-9)
    np.testing.assert_allclose(d, d[::-1], atol=1e-6)
    np.testing.assert_allclose(E, ctx.solve_chain(c), atol=1e-9 * np.abs(E).max())


def test_invalid_requests(ctx):
    with pytest.raises(P.RmcError) as e:
        ctx.solve_chain_states(I.tfim(25, 1.0, 0.9, 5, 8, 2), states=True)
    assert e.value.status == P.RMC_ERR_INVAL
    with pytest.raises(P.RmcError) as e:
        ctx.solve_chain_states(I.tfim(8, 1.0, 0.9, 4, 8, 2), observables=[(8, "X")])
    assert e.value.status == P.RMC_ERR_INVAL
