"""The oracle's pins catch planted mistakes (CPU only).

Each case swaps the oracle's loop body for a copy that carries one plausible
mistake, or the SVT for a variant, and runs the pins that exercise it. At least
one pin must fail, by an assertion or an error. The unmutated copy passes every
pin (the control case), so each failure comes from the planted mistake alone.
This checks the pins themselves; the CUDA path is not involved.
"""
import numpy as np
import pytest

from oracle import pasd_oracle as O
import test_oracle_pins as pins


def _step_with(kind):
    """A copy of the oracle's loop body (Algorithm 1) with the mistake `kind`."""

    def step(T, st, p):
        dims = T.shape
        n_modes = len(dims)
        mu = st.mu
        y_sign = -1.0 if kind == "y_sign" else 1.0
        mu_y = p.rho * mu if kind == "mu_before_y" else mu
        new_u, new_v, new_null, zs = [], [], [], []
        kept, sig, nuc, amats = [], [], [], []
        for n in range(n_modes):
            g = O.unfold(T - st.E + y_sign * st.Y[n] / mu, n)
            m = g @ st.V[n].T
            null = np.zeros((p.ranks[n], 0)) if kind == "null_dropped" else st.null[n]
            u = O.procrustes(m, st.U[n], null)
            a = (st.U[n] if kind == "a_old_u" else u).T @ g
            scale = 2.0 if kind == "svt_threshold" else 1.0
            sv = O.svt(a, scale * p.lambdas[n] / mu)
            v = np.roll(sv.V, 1, axis=1) if kind == "v_shift" else sv.V
            new_u.append(u)
            new_v.append(v)
            new_null.append(sv.left[:, sv.kept:])
            zs.append(O.fold(u @ v, n, dims))
            kept.append(sv.kept)
            sig.append(sv.sigma)
            nuc.append(sv.nuclear)
            amats.append(a)
        h_mean = sum(T - zs[n] + st.Y[n] / mu for n in range(n_modes)) / n_modes
        e_tau = 1.0 / mu if kind == "e_threshold" else 1.0 / (mu * n_modes)
        e = O.soft_threshold(h_mean, e_tau)
        res_inf, res_fro, new_y = 0.0, 0.0, []
        for n in range(n_modes):
            r = T - zs[n] - e
            new_y.append(st.Y[n] + mu_y * r)
            res_inf = max(res_inf, float(np.max(np.abs(r))))
            res_fro = max(res_fro, float(np.linalg.norm(r)))
        t_norm = float(np.linalg.norm(T))
        st.U, st.V, st.null, st.E, st.Y = new_u, new_v, new_null, e, new_y
        st.mu = min(p.rho * mu, p.mu_max)
        st.k += 1
        obj = sum(l * v for l, v in zip(p.lambdas, nuc)) + float(np.abs(e).sum())
        return O.StepInfo(kept=kept, sigma=sig, nuclear=nuc, A=amats, Z=zs, res_inf=res_inf,
                          res_fro_rel=res_fro / t_norm if t_norm > 0 else 0.0, objective=obj, mu_used=mu)

    return step


def _svt_keeping_ties(x, tau):
    """The SVT with `>=` in place of `>`: a singular value equal to tau is kept."""
    u, s, vt = np.linalg.svd(x, full_matrices=x.shape[0] > x.shape[1])
    if x.shape[0] > x.shape[1]:
        vt = vt[:x.shape[1]]
        s = np.concatenate([s, np.zeros(x.shape[0] - x.shape[1])])
    shrunk = np.maximum(s - tau, 0.0)
    kept = int(np.count_nonzero(s >= tau))
    v = (u[:, :kept] * shrunk[:kept]) @ vt[:kept, :]
    return O.SvtOut(V=v, left=u, sigma=s, kept=kept, nuclear=float(shrunk.sum()))


PINS = [
    ("horpca", lambda: pins.test_full_rank_bound_reduces_to_horpca((6, 5, 4), (2, 2, 2))),
    ("eqS1", pins.test_multiplier_sum_bound_eqS1),
    ("eqS3", pins.test_dual_spectral_bound_eqS3),
    ("idle", pins.test_idle_phase_matches_closed_form),
    ("svt_tie", pins.test_svt_drops_a_singular_value_equal_to_tau),
    ("alpha_output", pins.test_output_is_the_alpha_weighted_mean_of_the_refolds),
]


def _failing_pins(monkeypatch, step=None, svt=None, output=None, stop_at_first=True):
    if step is not None:
        monkeypatch.setattr(O, "step", step)
    if svt is not None:
        monkeypatch.setattr(O, "svt", svt)
    if output is not None:
        monkeypatch.setattr(O, "output_low_rank", output)
    failed = []
    for name, pin in PINS:
        try:
            pin()
        except Exception:   # an assertion or an error inside the mutated iteration
            failed.append(name)
            if stop_at_first:
                break
    return failed


def test_unmutated_copy_passes_every_pin(monkeypatch):
    assert _failing_pins(monkeypatch, step=_step_with("none"), stop_at_first=False) == []


@pytest.mark.parametrize("kind", ["e_threshold", "svt_threshold", "mu_before_y", "y_sign", "a_old_u",
                                  "v_shift", "null_dropped"])
def test_a_planted_mistake_in_the_body_fails_a_pin(monkeypatch, kind):
    assert _failing_pins(monkeypatch, step=_step_with(kind))


def test_keeping_svt_ties_fails_a_pin(monkeypatch):
    assert _failing_pins(monkeypatch, svt=_svt_keeping_ties)


def _output_ignoring_alpha(zs, alpha):
    """Algorithm 1's output with the weights dropped: the plain mean of the Z_n."""
    return sum(zs) / len(zs)


def _output_unnormalised(zs, alpha):
    """Algorithm 1's output without the division by sum_n alpha_n."""
    alpha = [1.0 / len(zs)] * len(zs) if alpha is None else alpha
    return sum(a * z for a, z in zip(alpha, zs))


@pytest.mark.parametrize("output", [_output_ignoring_alpha, _output_unnormalised])
def test_a_planted_mistake_in_the_output_fails_a_pin(monkeypatch, output):
    assert _failing_pins(monkeypatch, output=output)
