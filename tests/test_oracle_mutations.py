"""Planted mistakes in the oracle: each one must make one of its pins fail.

The pins in tests/test_oracle_*.py are chosen so that a plausible mistake anywhere in the oracle
(a dropped term, a wrong sign, index or digit order, a transposed operand, the other bond
flattening, a threshold off by a factor) fails one of them.  This module checks that claim: each
case builds a copy of one oracle function from its own source with one such mistake (one textual
change, applied on the CPU; the oracle's files are untouched), puts it in place of the original
for the duration of the case, runs the pins that cover that function and requires at least one
of them to fail an assertion.  A pin that errors out on the mutant (a shape mismatch) does not
count: every mutant keeps the shapes valid, so the mistake can only show in the values.

Several cases plant a reading that the oracle rejects on purpose: the paper's printed middle core
of the polynomial TT (bond indices transposed, Section 4.1) and a threshold without the
1/sqrt(L - 1) of the per-bond budget.
"""
import inspect
import textwrap

import pytest

from oracle import approx, core, grad, qft, structured

import test_oracle_approx as pa
import test_oracle_exact as pe
import test_oracle_grad as pg
import test_oracle_qft as pq
import test_oracle_round as pr
import test_oracle_structured as ps


def _mutant(module, name, old, new):
    """The function `name` of `module`, recompiled from its source with `old` replaced by `new`
    (which must occur exactly once), in a copy of the module's namespace."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, (module.__name__, name, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<{module.__name__}.{name}, planted mistake>", "exec"), ns)
    return ns[name]


# (case id, module, function, text in the oracle, planted text, pins that must catch it)
CASES = [
    # ---- exact operations (Sections 2 and 3.1)
    ("apply_mpo: input bond major", core, "apply_mpo",
     '"aijb,rjs->aribs"', '"aijb,rjs->raisb"',
     [pe.test_apply_mpo_bond_flatten_operator_major]),
    ("apply_mpo: operator transposed", core, "apply_mpo",
     '"aijb,rjs->aribs"', '"ajib,rjs->aribs"',
     [lambda: pe.test_apply_mpo_is_matvec([2] * 8)]),
    ("hadamard: second operand major", core, "hadamard",
     '"ria,sib->rsiab"', '"ria,sib->sriba"',
     [pe.test_hadamard_flatten_first_operand_major]),
    ("add: B in the off-diagonal block", core, "add",
     "c[ra0:, :, ra1:] = b", "c[ra0:, :, :rb1] = b",
     [lambda: pe.test_add_block_sum([2] * 7)]),
    ("add: first core [B A]", core, "add",
     "c[:, :, :ra1] = a\n            c[:, :, ra1:] = b", "c[:, :, :rb1] = b\n            c[:, :, rb1:] = a",
     [lambda: pe.test_add_block_sum([2] * 7)]),
    ("inner: digits of y reversed", core, "inner",
     'np.einsum("ab,aic,bid->cd", e, xk, yk, optimize=True)',
     'np.einsum("ab,aic,bid->cd", e, xk, yk[:, ::-1, :], optimize=True)',
     [pe.test_inner_and_norm_brute_force, pe.test_inner_closed_form_exponentials]),
    ("evaluate: sites read last to first", core, "evaluate",
     "digits[:, k].astype(np.int64)", "digits[:, len(x) - 1 - k].astype(np.int64)",
     [lambda: pe.test_evaluate_brute_force([2] * 10)]),
    ("rel_err: divided by ||a||", core, "rel_err",
     "return nd / nb if nb > 0 else nd", "return nd / norm(a) if nb > 0 else nd",
     [pe.test_rel_err_brute_force]),
    # ---- orthogonalisation and rounding (Section 3.2)
    ("orthogonalize_rl: Q not transposed back", core, "orthogonalize_rl",
     "np.ascontiguousarray(q.T).reshape(p, d, r1)", "np.ascontiguousarray(q).reshape(p, d, r1)",
     [pr.test_orthogonalize_keeps_tensor_and_orthonormalises, pr.test_norm_from_first_core]),
    ("norm: first core without the sweep", core, "norm",
     "c = orthogonalize_rl(x)", "c = [np.asarray(g) for g in x]",
     [pr.test_norm_from_first_core, pe.test_inner_and_norm_brute_force]),
    ("round_tt: threshold without 1/sqrt(L-1)", core, "round_tt",
     "delta = eps * nrm / math.sqrt(L - 1)", "delta = eps * nrm",
     [lambda: pr.test_round_known_bond_spectrum(5), lambda: pr.test_rounding_bound(1e-1)]),
    ("round_tt: S dropped from the carried factor", core, "round_tt",
     "sv = s[:rn, None] * vt[:rn]", "sv = vt[:rn]",
     [pr.test_round_redundant_ranks_exact]),
    ("round_tt: trailing singular vectors kept", core, "round_tt",
     "(q @ u[:, :rn])", "(q @ u[:, u.shape[1] - rn:])",
     [lambda: pr.test_rounding_bound(1e-1), pr.test_round_two_sites_is_truncated_svd]),
    ("round_tt: norm of the unswept first core", core, "round_tt",
     "nrm = float(np.linalg.norm(c[0]))", "nrm = float(np.linalg.norm(x[0]))",
     [lambda: pr.test_round_known_bond_spectrum(5), lambda: pr.test_rounding_bound(1e-1)]),
    ("truncation_rank: exclusive tail bound", core, "truncation_rank",
     "if math.sqrt(t) <= delta:", "if math.sqrt(t) < delta:",
     [pr.test_truncation_rank_rule]),
    ("truncation_rank: tail of sigma, not sigma^2", core, "truncation_rank",
     "t = tail2 + sigma[j] * sigma[j]", "t = tail2 + sigma[j]",
     [pr.test_truncation_rank_rule, pr.test_round_two_sites_is_truncated_svd]),
    # ---- structured tensors and operators (Section 4)
    ("coefficients: least significant digit first", structured, "coefficients",
     "    return c\n", "    return c[::-1]\n",
     [pe.test_quantization_digits_roundtrip, lambda: ps.test_exp_closed_form([2, 3, 5, 2, 3])]),
    ("exp_tt: offset e^{v(a - x0)} dropped", structured, "exp_tt",
     "vals = vals * math.exp(v * (lower - x0))", "vals = vals",
     [lambda: ps.test_exp_closed_form([2] * 10)]),
    ("cos_tt: sign of the rotation", structured, "cos_tt",
     "rot[0, :, 1] = -np.sin(t)", "rot[0, :, 1] = np.sin(t)",
     [lambda: ps.test_cos_sin_closed_form([2] * 12)]),
    ("poly_tt: middle core as printed (bonds transposed)", structured, "poly_tt",
     "c[s, :, u] = binom[s][u] * t ** (s - u)", "c[u, :, s] = binom[s][u] * t ** (s - u)",
     [lambda: ps.test_polynomial_closed_form([0.3, -1.0, 0.5, 2.0, -0.7])]),
    ("shift_mpo: carry blocks swapped", structured, "shift_mpo",
     "blocks = [[q_shift(b, dq[q]), q_shift(b, dq[q] + 1)],", "blocks = [[q_shift(b, dq[q] + 1), q_shift(b, dq[q])],",
     [lambda: ps.test_shift_mpo_is_shift_matrix([2] * 6, 13), ps.test_shift_cores_golden]),
    ("r_shift: not transposed", structured, "r_shift",
     "q_shift(b, b - d).T", "q_shift(b, b - d)",
     [lambda: ps.test_shift_mpo_is_shift_matrix([2, 3, 5], 7), ps.test_shift_cores_golden]),
    ("shift_digits: digit of the remainder not removed", structured, "shift_digits",
     "rem -= out[-1] * cq", "rem -= out[-1]",
     [lambda: ps.test_shift_mpo_is_shift_matrix([2] * 6, 13)]),
    ("digit values: spacing (b - a)/N instead of (b - a)/(N - 1)", structured, "_digit_values",
     "h = (upper - lower) / (n_total - 1)", "h = (upper - lower) / n_total",
     [lambda: ps.test_exp_closed_form([2] * 10)]),
    ("mpo_add: second operator in the off-diagonal block", structured, "mpo_add",
     "c[ra0:, :, :, ra1:] = b", "c[ra0:, :, :, :rb1] = b",
     [lambda: ps.test_laplacian_dense(1, 8, 3)]),
    ("interleaved_layout: all bits of x first", structured, "interleaved_layout",
     "[k % n_dims for k in range(n_dims * bits)]", "[k // bits for k in range(n_dims * bits)]",
     [lambda: ps.test_laplacian_dense(2, 4, 5)]),
    ("second difference: +2I", structured, "second_difference_sum_mpo",
     "mpo_scale(mpo_identity(bases), -2.0)", "mpo_scale(mpo_identity(bases), 2.0)",
     [lambda: ps.test_laplacian_dense(1, 8, 3)]),
    ("laplacian_mpo: + and - carries swapped at the last site", structured, "laplacian_mpo",
     'c[idx[(owner, "+")], :, :, idx["done"]] = Jt', 'c[idx[(owner, "+")], :, :, idx["done"]] = J',
     [ps.test_second_difference_small_dense, lambda: ps.test_laplacian_dense(1, 8, 3)]),
    ("laplacian_mpo: pending terms of other dimensions dropped", structured, "laplacian_mpo",
     "if pending_other:", "if False:",
     [lambda: ps.test_laplacian_dense(2, 4, 5)]),
    # ---- approximate einsums (Section 3.2 zip-up, Section 3.3 variational fit)
    ("zip-up: threshold without 1/sqrt(L-1)", approx, "decomposition_apply",
     "delta = eps * float(np.linalg.norm(sc)) / math.sqrt(L - 1)", "delta = eps * float(np.linalg.norm(sc))",
     [lambda: pa.test_decomposition_over_the_whole_train_is_the_rounding(1e-1)]),
    ("zip-up: S kept on the split-off core", approx, "decomposition_apply",
     "out.append(u[:, :rn].reshape(left, d, rn))\n        sc = (s[:rn, None] * vt[:rn])",
     "out.append((u[:, :rn] * s[None, :rn]).reshape(left, d, rn))\n        sc = (vt[:rn])",
     [lambda: pa.test_decomposition_over_the_whole_train_is_the_rounding(1e-1)]),
    ("variational: left environment with the digits of y reversed", approx, "_left_env",
     'np.einsum("ab,aic,bid->cd", e, c[p], y[p], optimize=True)',
     'np.einsum("ab,aic,bid->cd", e, c[p], y[p][:, ::-1, :], optimize=True)',
     [lambda: pa.test_variational_centre_is_the_overlap_gradient(1),
      lambda: pa.test_variational_updates_never_increase_the_distance(1, 4)]),
    ("variational: updated core kept instead of its orthonormal Q", approx, "variational_apply",
     "c[q] = qm.reshape(r0, d, qm.shape[1])", "c[q] = c[q].reshape(r0, d, r1)",
     [lambda: pa.test_variational_centre_is_the_overlap_gradient(1),
      lambda: pa.test_variational_updates_never_increase_the_distance(1, 4)]),
    ("variational: S left on the left core when sweeping right", approx, "variational_apply",
     "c[q] = u[:, :rn].reshape(r0, d0, rn)\n            c[q + 1] = (s[:rn, None] * vt[:rn]).reshape(rn, d1, r1)",
     "c[q] = (u[:, :rn] * s[None, :rn]).reshape(r0, d0, rn)\n            c[q + 1] = vt[:rn].reshape(rn, d1, r1)",
     [lambda: pa.test_variational_centre_is_the_overlap_gradient(2),
      lambda: pa.test_variational_updates_never_increase_the_distance(2, 4)]),
    # ---- the Fourier tensor train (Section 4.3)
    ("fourier factors: column digits not reversed", qft, "_weights",
     "w = [int(np.prod(bases[:p], dtype=np.int64)) for p in range(n)]", "w = list(c)",
     [lambda: pq.test_exact_product_is_the_fft([3, 2, 2, 5, 2, 2])]),
    ("fourier factor: delta(s, i_q) dropped", qft, "factor_mpo",
     "g[s, s, jp, s] = phase", "g[s, :, jp, s] = phase",
     [lambda: pq.test_factor_mpos_are_rank_bq_phases([3, 2, 2, 5, 2, 2])]),
    ("fourier factor: exponent without the row weight c_q", qft, "factor_mpo",
     "(s * c[q] * w[p] * jp) % N", "(s * w[p] * jp) % N",
     [lambda: pq.test_factor_mpos_are_rank_bq_phases([3, 2, 2, 5, 2, 2])]),
    ("dft matrix: v = exp(+2 pi i / N)", qft, "dft_rows",
     "table = np.exp(-2j * np.pi", "table = np.exp(2j * np.pi",
     [pq.test_paper_distances_n8192]),
    # ---- adjoints (Section 3.3 environments; the reverse of the rounding sweeps)
    ("apply_mpo_vjp: dW with i and j swapped", grad, "apply_mpo_vjp",
     '"rjs,aribs->aijb"', '"rjs,aribs->ajib"',
     [pg.test_apply_vjp_fd]),
    ("hadamard_vjp: dZ read second operand major", grad, "hadamard_vjp",
     "d5 = dzk.reshape(r0, s0, d, r1, s1)", "d5 = dzk.reshape(s0, r0, d, s1, r1).transpose(1, 0, 2, 4, 3)",
     [pg.test_hadamard_vjp_fd]),
    ("inner_vjp: digits of y reversed in dX", grad, "inner_vjp",
     'np.einsum("ab,bid,cd->aic", el, y[k], er, optimize=True)',
     'np.einsum("ab,bid,cd->aic", el, y[k][:, ::-1, :], er, optimize=True)',
     [pg.test_inner_vjp_fd, pg.test_inner_vjp_brute_force]),
    ("evaluate_vjp: sample weights dropped", grad, "evaluate_vjp",
     'np.einsum("s,sa,sb->sab", dv, pre[k], suf[k + 1])', 'np.einsum("sa,sb->sab", pre[k], suf[k + 1])',
     [pg.test_evaluate_vjp_fd]),
    ("evaluate_vjp: samples grouped by the next site's digit", grad, "evaluate_vjp",
     "m = digits[:, k] == i", "m = digits[:, (k + 1) % L] == i",
     [pg.test_evaluate_vjp_fd]),
    ("fit_loss_grad: residual not divided by the sample count", grad, "fit_loss_grad",
     "(v - targets) / n)", "(v - targets))",
     [pg.test_fit_loss_grad_fd]),
    ("residual_loss_grad: sign of the <y, b> term", grad, "residual_loss_grad",
     "inner_vjp(y, b, -2.0)", "inner_vjp(y, b, 2.0)",
     [pg.test_residual_loss_grad_fd]),
    ("residual_loss_grad: one slot of <y, y> only", grad, "residual_loss_grad",
     "a + c + e for", "a + e for",
     [pg.test_residual_loss_grad_fd]),
    ("copyltu: upper triangle copied down", grad, "_copyltu",
     "lo = np.tril(m)\n    return lo + np.tril(m, -1).T", "lo = np.triu(m)\n    return lo + np.triu(m, 1).T",
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-8)]),
    ("qr_vjp: copyltu term dropped", grad, "_qr_vjp",
     "rhs = dq + q @ _copyltu(mm)", "rhs = dq",
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-8)]),
    ("qr_vjp: Y dR2^T term of the wide case dropped", grad, "_qr_vjp",
     "dq + y @ dr2.T, dr1", "dq, dr1",
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-8)]),
    ("left_vectors_vjp: sign of the gap s_j^2 - s_i^2", grad, "_left_vectors_vjp",
     "diff = s2[None, :] - s2[:, None]", "diff = s2[:, None] - s2[None, :]",
     [lambda: pg.test_round_vjp_fd(1e-3), pg.test_round_vjp_fd_norm_loss]),
    ("left_vectors_vjp: projection I - u u^T dropped", grad, "_left_vectors_vjp",
     "x = db - u @ (u.T @ db)", "x = db",
     [lambda: pg.test_round_vjp_fd(1e-3), pg.test_round_vjp_fd_norm_loss]),
    ("left_vectors_vjp: S_r^-1 in place of S_r^-2", grad, "_left_vectors_vjp",
     "1.0 / np.where(sr > 0.0, sr * sr, 1.0)", "1.0 / np.where(sr > 0.0, sr, 1.0)",
     [lambda: pg.test_round_vjp_fd(1e-3), pg.test_round_vjp_fd_norm_loss]),
    ("round_vjp: B dF term dropped", grad, "round_vjp",
     "da = b @ df + _left_vectors_vjp", "da = _left_vectors_vjp",
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-3)]),
    ("round_vjp: cotangent of the next core not carried", grad, "round_vjp",
     "dcrl[k + 1] = (f.T @ gm).reshape(n1, d1, r2)", "dcrl[k + 1] = 0.0 * nxt",
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-3)]),
    ("round_vjp: dR of the right-to-left factors dropped", grad, "round_vjp",
     'drr = np.einsum("adp,adb->pb", dd, xprev)', 'drr = 0.0 * rr',
     [pg.test_round_vjp_without_truncation_is_the_inner_gradient, lambda: pg.test_round_vjp_fd(1e-8)]),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _, module, name, old, new, pins = case
    monkeypatch.setattr(module, name, _mutant(module, name, old, new))
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError as e:
            caught.append(e)
    assert caught, "no pin failed"


def test_unplanted_copies_pass_their_pins(monkeypatch):
    """The same recompilation with no change leaves every pin green (so a failure above comes
    from the planted mistake, not from recompiling the function)."""
    seen = set()
    for _, module, name, old, _, pins in CASES:
        if (module, name) in seen:
            continue
        seen.add((module, name))
        with monkeypatch.context() as m:
            m.setattr(module, name, _mutant(module, name, old, old))
            for pin in pins:
                pin()
