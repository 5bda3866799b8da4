"""Planted mistakes: each pin of the oracle must be able to fail.

A plausible slip is planted in a throwaway copy of an oracle source (the C
operator and clover term, the numpy FGMRES-DR, CGNE and HMC routines), the
copy is compiled or executed on the CPU, and the existing pins are run
against it: every mutation must make at least one pin fail.  The committed
oracle itself is never changed.

C mutations (the operator and the clover term):
  projector sign    (1 - g_mu) and (1 + g_mu) exchanged on every hop;
  clover i-factor   c_sw (1/4) sigma F instead of c_sw (i/4) sigma F;
  leaf orientation  the first clover leaf traversed clockwise;
  boundary sign     the boundary sign put on the hop out of x_mu = 0 instead of
                    the one that wraps from x_mu = L_mu - 1.
FGMRES-DR: the harmonic-Ritz system solved with H_m instead of H_m^H, the
residual coordinates c + Hbar y instead of c - Hbar y, and the k largest
instead of the k smallest harmonic Ritz values kept.
CGNE: the step length, the residual update or the direction update mutated.
HMC: the gauge force's sign flipped, the fermion force's factor 2 dropped, a
full instead of a half final momentum step.
"""
import ctypes
import inspect
import os
import subprocess
import types

import pytest

import test_oracle_cgne as pins_cgne
import test_oracle_dirac as pins_dirac
import test_oracle_fgmres_dr as pins_dr
import test_oracle_hmc as pins_hmc

ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

LEAF0 = """        h[0] = (hop){i, mu, 0};
        h[1] = (hop){shift(L, i, mu, 1), nu, 0};
        h[2] = (hop){shift(L, i, nu, 1), mu, 1};
        h[3] = (hop){i, nu, 1};"""
LEAF0_CLOCKWISE = """        h[0] = (hop){i, nu, 0};
        h[1] = (hop){shift(L, i, nu, 1), mu, 0};
        h[2] = (hop){shift(L, i, mu, 1), nu, 1};
        h[3] = (hop){i, mu, 1};"""

C_MUTATIONS = {
    "projector sign": ("v += sgn * GAM[mu][s][t] * in[t * 3 + c];", "v -= sgn * GAM[mu][s][t] * in[t * 3 + c];"),
    "clover i-factor": ("csw * 0.25 * I * sg * F[mu][nu].m[a][b]", "csw * 0.25 * sg * F[mu][nu].m[a][b]"),
    "leaf orientation": (LEAF0, LEAF0_CLOCKWISE),
    "boundary sign": ("return (x[mu] == L[mu] - 1) ? bc[mu] : 1.0;", "return (x[mu] == 0) ? bc[mu] : 1.0;"),
}


def _mutated_source(src, old, new):
    assert src.count(old) == 1, "the mutation site must exist exactly once: %r" % old
    return src.replace(old, new)


def _failures(calls):
    """Run pin callables; return the names of those that fail (AssertionError)."""
    failed = []
    for name, fn in calls:
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def _dirac_pins(orc):
    return [
        ("plane wave", lambda: pins_dirac.test_free_field_plane_wave(orc, (4, 2, 4, 6))),
        ("gamma5 hermiticity", lambda: pins_dirac.test_gamma5_hermiticity(orc)),
        ("clover hermitian, chiral", lambda: pins_dirac.test_clover_hermitian_and_chiral(orc)),
        ("gauge covariance", lambda: pins_dirac.test_gauge_covariance(orc)),
        ("dense assembly", lambda: pins_dirac.test_dense_assembly(orc, (2, 2, 2, 2), pins_dirac.AP)),
        ("abelian clover (1,2)", lambda: pins_dirac.test_clover_abelian_closed_form(orc, (1, 2), (4, 8, 4, 2),
                                                                                    (1, -1, 1, -1))),
    ]


def test_unmutated_oracle_passes_the_pins(orc):
    """The control: with the committed oracle every pin above passes."""
    assert _failures(_dirac_pins(orc)) == []


@pytest.mark.parametrize("mutation", sorted(C_MUTATIONS))
def test_c_oracle_mutation_fails_a_pin(orc, mutation, tmp_path, monkeypatch):
    with open(ORACLE_C) as f:
        src = f.read()
    old, new = C_MUTATIONS[mutation]
    path_c = tmp_path / "oracle_mut.c"
    path_c.write_text(_mutated_source(src, old, new))
    path_so = str(tmp_path / "liboracle_mut.so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", str(path_c), "-o", path_so,
                           "-lm"])
    monkeypatch.setattr(orc, "_lib", orc.bind(ctypes.CDLL(path_so)))
    failed = _failures(_dirac_pins(orc))
    assert failed, "no pin caught the planted %s" % mutation


def _mutated_module(module, old, new):
    src = _mutated_source(inspect.getsource(module), old, new)
    mod = types.ModuleType(module.__name__ + "_mutated")
    mod.__file__ = module.__file__
    exec(compile(src, module.__file__ + " (mutated)", "exec"), mod.__dict__)
    return mod


DR_MUTATIONS = {
    "harmonic Ritz system transposed": ("f = np.linalg.solve(Hm.conj().T, em)", "f = np.linalg.solve(Hm, em)"),
    "residual coordinates sign": ("s = c - H @ y", "s = c + H @ y"),
    "largest Ritz values kept": ("order = np.argsort(np.abs(theta))[:k]", "order = np.argsort(-np.abs(theta))[:k]"),
}


@pytest.mark.parametrize("mutation", sorted(DR_MUTATIONS))
def test_fgmres_dr_mutation_fails_a_pin(orc, mutation, monkeypatch):
    import oracle.fgmres_dr as dr
    mod = _mutated_module(dr, *DR_MUTATIONS[mutation])
    monkeypatch.setattr(dr, "fgmres_dr", mod.fgmres_dr)
    failed = _failures([
        ("Arnoldi relation after a deflated restart", lambda: pins_dr.test_arnoldi_relation_after_deflated_restart(orc)),
        ("harmonic Ritz values of a known spectrum", pins_dr.test_harmonic_ritz_values_find_the_small_eigenvalues),
    ])
    assert failed, "no pin caught the planted %s" % mutation


CG_MUTATIONS = {
    "step length": ("alpha = rr / np.vdot(t, t).real", "alpha = rr / np.vdot(p, p).real"),
    "residual update": ("r = r - alpha * Dh(t)", "r = r - alpha * t"),
    "direction update": ("p = r + (rr_new / rr) * p", "p = r + (rr / rr_new) * p"),
}


@pytest.mark.parametrize("mutation", sorted(CG_MUTATIONS))
def test_cgne_mutation_fails_a_pin(orc, mutation, monkeypatch):
    import oracle.cgne as cg
    mod = _mutated_module(cg, *CG_MUTATIONS[mutation])
    monkeypatch.setattr(cg, "cgne", mod.cgne)
    failed = _failures([
        ("orthogonal residuals", lambda: pins_cgne.test_residuals_are_orthogonal(orc)),
        ("finite termination", pins_cgne.test_finite_termination_on_small_spectrum),
    ])
    assert failed, "no pin caught the planted %s" % mutation


HMC_MUTATIONS = {
    "gauge force sign": ("return (beta / 6.0) * np.einsum", "return -(beta / 6.0) * np.einsum"),
    "fermion force factor": ("F[x, mu, a] = -2.0 * np.vdot(Y, dDX).real", "F[x, mu, a] = -1.0 * np.vdot(Y, dDX).real"),
    "full final momentum step": ("step = eps if s < nsteps - 1 else 0.5 * eps", "step = eps"),
}
HMC_PIN = {
    "gauge force sign": lambda orc, inputs: pins_hmc.test_gauge_force_matches_finite_difference(),
    "fermion force factor": lambda orc, inputs: pins_hmc.test_fermion_force_matches_finite_difference(orc),
    "full final momentum step": lambda orc, inputs: pins_hmc.test_trajectory_is_reversible(orc, inputs),
}


@pytest.mark.slow
@pytest.mark.parametrize("mutation", sorted(HMC_MUTATIONS))
def test_hmc_mutation_fails_its_pin(orc, mutation, monkeypatch):
    import oracle
    import oracle.hmc
    from paper_1109_4279_gb300 import synth
    mod = _mutated_module(oracle.hmc, *HMC_MUTATIONS[mutation])
    monkeypatch.setattr(oracle, "hmc", mod)
    U, rng = synth.gauge_field(pins_hmc.DIMS, 0.3, 11)
    inputs = (U, rng.standard_normal((pins_hmc.V, 4, 8)), synth.gaussian_spinor(pins_hmc.DIMS, rng))
    with pytest.raises(AssertionError):
        HMC_PIN[mutation](orc, inputs)
