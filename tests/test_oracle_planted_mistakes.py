"""Planted mistakes in the oracle: each case edits one line of one oracle function (a
flipped sign, a dropped term or factor, a transposed operand, a wrong index, axis or
cutoff) in a copy of that function, installs the copy wherever the oracle binds the
original for the length of the case, and runs the pins that should notice.  A case
passes only when one of its pins fails.  The pins compare the oracle with things
other than itself (dense matrices written from the DFT's sum, closed forms, LAPACK
least squares, the assembled sparse matrices, finite differences, numpy's FFT), so
these cases show that a plausible slip on each of these lines does not go unseen.
Edits are made on the CPU, to the oracle only, and undone after each case.

Edits that turned out to give the same results as the original are not listed as
mistakes: reversing the axes of the Green's function block (the kernel is symmetric
under axis swaps on a square grid), conjugating the second argument of the Givens
rotation (it is always the real norm of the new Arnoldi vector), and transposing R in
the network's mode mixing in both passes (a relabelling of the parameters).
"""
import __future__
import inspect
import sys
import textwrap

import pytest

import oracle
import oracle.fno as FN
import oracle.gmres as GM
import oracle.precond as PR
import oracle.spectral as SP
import oracle.stencil as ST
import test_fno_oracle as TF
import test_oracle_sampled_rows as TSr
import test_oracle_solve as TSo
import test_oracle_spectral as TSp
import test_oracle_stencil as TSt
import test_stencil_pointwise as TPw

_PINV_CUTOFF = (ST, "matlab_pinv", "tol = max(B.shape)", "tol = min(B.shape)")

# (id, module, function, line as written, planted line, pins, what the failing pin raises)
CASES = [
    ("green_symbol_sign", SP, "green_symbol", "den = laplacian_symbol(d, n) - s",
     "den = laplacian_symbol(d, n) + s",
     [lambda: TSp.test_green_apply_matches_dense_definition(2, 4)], AssertionError),
    ("wavenumbers_unscaled", SP, "wavenumber_grid", "np.fft.fftfreq(n, d=1.0 / n)",
     "np.fft.fftfreq(n)", [lambda: TSp.test_plane_wave_closed_form(2, 16, (3, -5))], AssertionError),
    ("operator_drops_identity", SP, "apply_operator",
     "return x + apply_green(d, n, s, np.asarray(q) * x)",
     "return apply_green(d, n, s, np.asarray(q) * x)",
     [TSp.test_integral_reformulation_identity], AssertionError),
    ("operator_q_after_G", SP, "apply_operator",
     "return x + apply_green(d, n, s, np.asarray(q) * x)",
     "return x + np.asarray(q) * apply_green(d, n, s, x)",
     [TSp.test_integral_reformulation_identity], AssertionError),
    ("helmholtz_split_sign", SP, "helmholtz_shift", "return s, (s - w2c2).ravel()",
     "return s, (w2c2 - s).ravel()", [TSp.test_helmholtz_shift_split], AssertionError),
    ("schrodinger_energy_unscaled", SP, "schrodinger_shift",
     "pot = l2 * np.asarray(V, dtype=np.float64) - l2 * E",
     "pot = l2 * np.asarray(V, dtype=np.float64) - E",
     [TSp.test_schrodinger_shift_split], AssertionError),
    ("green_kernel_forward_fft", SP, "green_kernel", "np.fft.ifftn(green_symbol(d, n, s)).real",
     "np.fft.fftn(green_symbol(d, n, s)).real",
     [TSp.test_green_kernel_is_the_convolution_kernel], AssertionError),
    ("gamma_one_short", ST, "canonical_gamma", "list(range(0, b + 1))", "list(range(0, b))",
     [lambda: TSt.test_sets_partition_the_grid(2, 8, 2)], AssertionError),
    ("set_type_axis_reversed", ST, "canonical_set", "[0] if (t >> a) & 1",
     "[0] if (t >> (d - 1 - a)) & 1",
     [lambda: TSt.test_sets_partition_the_grid(2, 8, 2)], AssertionError),
    ("flat_index_axes_reversed", ST, "flat_index", "pts[:, a] * n ** a",
     "pts[:, a] * n ** (pts.shape[1] - 1 - a)",
     [lambda: TSt.test_C_is_QG_on_the_pattern_and_P(2, 16, 4)], AssertionError),
    ("Q_sign_of_T", ST, "_q_and_c", "= -T", "= T",
     [lambda: TSt.test_C_is_QG_on_the_pattern_and_P(2, 16, 4)], AssertionError),
    ("green_block_sum_of_points", ST, "green_block", "np.mod(rows[r][None, :] - col_pts, n)",
     "np.mod(rows[r][None, :] + col_pts, n)",
     [lambda: TSt.test_C_is_QG_on_the_pattern_and_P(2, 16, 4)], AssertionError),
    ("T_without_pinv", ST, "stencil_tables", "T = A @ Bp", "T = A @ B.T",
     [lambda: TSt.test_T_least_squares(2, 16, 4)], AssertionError),
    ("pinv_cutoff_min_dimension",) + _PINV_CUTOFF + ([TSt.test_matlab_pinv_truncation], AssertionError),
    ("pointwise_T_sign", ST, "pointwise_stencil_tables", "qrow[~centre] = -Tj",
     "qrow[~centre] = Tj", [TPw.test_pointwise_least_squares_pin], AssertionError),
    ("pointwise_C_without_Q", ST, "pointwise_stencil_tables",
     "crow = qrow @ green_block(g, n, gj, gj_flat)",
     "crow = green_block(g, n, p[None, :], gj_flat)[0]",
     [lambda: TPw.test_pointwise_C_is_QG_on_each_stencil(2, 16, 2)], AssertionError),
    ("pointwise_centre_misplaced", ST, "pointwise_stencil_tables",
     "centre = np.all(gj == p, axis=1)", "centre = np.all(gj == p + 1, axis=1)",
     [lambda: TPw.test_pointwise_structure_and_invariance(2, 16, 2, 1.37)], AssertionError),
    ("solve_P_imaginary_sign", PR, "SparsifyingPreconditioner.solve_P",
     "return sla.lu_solve(self._lu, y.real) + 1j * sla.lu_solve(self._lu, y.imag)",
     "return sla.lu_solve(self._lu, y.real) - 1j * sla.lu_solve(self._lu, y.imag)",
     [lambda: TSo.test_factorisation_independent_of_ordering(2, 16, 4)], AssertionError),
    ("apply_residual_sign", PR, "SparsifyingPreconditioner.apply_residual",
     "self.P @ np.asarray(z) - Qr", "self.P @ np.asarray(z) + Qr",
     [lambda: TSo.test_factorisation_independent_of_ordering(2, 16, 4)], AssertionError),
    ("P_scales_C_by_row_q", PR, "assemble_sparse", "Cv * np.asarray(q, dtype=np.float64)[cols]",
     "Cv * np.asarray(q, dtype=np.float64)[rows]",
     [lambda: TSt.test_C_is_QG_on_the_pattern_and_P(2, 16, 4)], AssertionError),
    ("P_rows_origin_reversed", PR, "assemble_sparse", "r = flat_index(S + o, n)",
     "r = flat_index(S + o[::-1], n)",
     [lambda: TSt.test_C_is_QG_on_the_pattern_and_P(2, 16, 4)], AssertionError),
    ("sampled_row_q_at_row", PR, "sampled_rows", "Qr + tab[\"C\"][a_idx] * q[cols]",
     "Qr + tab[\"C\"][a_idx] * q[j]",
     [lambda: TSr.test_rows_equal_assembled_matrices(2, 16, 4)], AssertionError),
    # a face point given to the lower box, or a type bit from the wrong residue: the
    # point is not in that set's canonical instance and the checker raises
    ("sampled_row_face_in_lower_box", PR, "sampled_rows", "o = (p // b) * b",
     "o = ((p - 1) // b) * b",
     [lambda: TSr.test_rows_equal_assembled_matrices(2, 16, 4)], IndexError),
    ("sampled_row_type_residue", PR, "sampled_rows", "if p[a] % b == 0", "if p[a] % b == 1",
     [lambda: TSr.test_rows_equal_assembled_matrices(2, 16, 4)], IndexError),
    ("sampled_residual_sign", PR, "sampled_apply_residual", "num += abs(pz - qr) ** 2",
     "num += abs(pz + qr) ** 2",
     [lambda: TSr.test_sampled_residual_equals_global(2, 16, 4)], AssertionError),
    ("gmres_update_without_M", GM, "gmres_right", "u = u + apply_M(V[:k].T @ y)",
     "u = u + V[:k].T @ y", [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gmres_rhs_rotation_sign", GM, "gmres_right", "gam[j + 1] = -np.conj(sn[j]) * gam[j]",
     "gam[j + 1] = np.conj(sn[j]) * gam[j]",
     [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gmres_old_rotation_sign", GM, "gmres_right",
     "H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]",
     "H[i + 1, j] = np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]",
     [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gmres_old_rotation_conjugate", GM, "gmres_right",
     "t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]",
     "t0 = cs[i] * H[i, j] + np.conj(sn[i]) * H[i + 1, j]",
     [lambda: TSo.test_gmres_minimal_residual_property(False, 6, 1e-9)], AssertionError),
    ("gram_schmidt_sign", GM, "gmres_right", "w = w - V[: j + 1].T @ c",
     "w = w + V[: j + 1].T @ c", [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gram_schmidt_no_conjugate", GM, "gmres_right", "c = V[: j + 1].conj() @ w",
     "c = V[: j + 1] @ w", [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gmres_history_index", GM, "gmres_right", "hist.append(abs(gam[j + 1]) / bnorm)",
     "hist.append(abs(gam[j]) / bnorm)",
     [TSo.test_counts_monotone_in_tolerance_and_history], AssertionError),
    ("givens_cosine_of_b", GM, "_givens", "c = abs(a) / r", "c = abs(b) / r",
     [TSo.test_gmres_equals_dense_pseudospectral_solve], AssertionError),
    ("gelu_scale", FN, "gelu", "erf(x / np.sqrt(2.0))", "erf(x / 2.0)",
     [TF.test_gelu_is_x_times_normal_cdf], AssertionError),
    ("gelu_prime_drops_x", FN, "gelu_prime", "x * np.exp(-0.5 * x * x)", "np.exp(-0.5 * x * x)",
     [TF.test_gelu_is_x_times_normal_cdf], AssertionError),
    ("negative_modes_shifted", FN, "ky_list", "np.arange(n - M, n)",
     "np.arange(n - M + 1, n + 1) % n", [TF.test_spectral_conv_is_truncated_rfft2], AssertionError),
    ("mix_transposed_forward_only", FN, "mix", "\"bikq,kqio->bokq\"", "\"bokq,kqio->bikq\"",
     [TF.test_gradient_matches_finite_differences], AssertionError),
    ("forward_drops_mode_doubling", FN, "forward", "1.0 / n**2, 2.0 / n**2",
     "1.0 / n**2, 1.0 / n**2", [TF.test_network_spectral_branch_is_truncated_irfft2],
     AssertionError),
    ("R_gradient_without_conjugate", FN, "backward",
     "G[f\"R{l}\"] = np.einsum(\"bokq,bikq->kqio\", dY, V.conj())",
     "G[f\"R{l}\"] = np.einsum(\"bokq,bikq->kqio\", dY, V)",
     [TF.test_gradient_matches_finite_differences], AssertionError),
    ("backward_mode_zero_weight", FN, "backward", "w[0] = 1.0 / n**2", "w[0] = 2.0 / n**2",
     [TF.test_gradient_matches_finite_differences], AssertionError),
    ("backward_gelu_on_last_layer", FN, "backward",
     "dh = dv * gelu_prime(h) if l < D.layers - 1 else dv", "dh = dv * gelu_prime(h)",
     [TF.test_gradient_matches_finite_differences], AssertionError),
    ("adam_no_second_moment_correction", FN, "adam_step", "vh = v / (1.0 - beta2**step)",
     "vh = v", [TF.test_adam_first_step_is_signed_lr], AssertionError),
    ("loss_gradient_not_batch_mean", FN, "loss",
     "dy = 2.0 * diff / (B * den[:, None, None, None])",
     "dy = 2.0 * diff / (den[:, None, None, None])",
     [TF.test_gradient_matches_finite_differences], AssertionError),
]


def _planted(module, name, line, planted):
    """A copy of module.name (a function, or "Class.method") with `line` replaced by
    `planted` (the line must occur once).  Returns (owner, attribute, original, copy)."""
    owner, attr = module, name
    if "." in name:
        cls, attr = name.split(".")
        owner = getattr(module, cls)
    fn = owner.__dict__[attr]
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(line) == 1, f"{module.__name__}.{name} no longer holds {line!r}"
    ns = dict(module.__dict__)
    code = compile(src.replace(line, planted), module.__file__, "exec",
                   __future__.annotations.compiler_flag, True)
    exec(code, ns)
    return owner, attr, fn, ns[attr]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _, module, name, line, planted, pins, raised = case
    owner, attr, orig, bad = _planted(module, name, line, planted)
    if owner is module:
        bound = [m for mn, m in list(sys.modules.items())
                 if (mn == "oracle" or mn.startswith("oracle.")) and getattr(m, attr, None) is orig]
        assert module in bound
    else:
        bound = [owner]  # a method: every module reaches it through the one class object
    for m in bound:
        monkeypatch.setattr(m, attr, bad)
    failed = []
    for pin in pins:
        try:
            pin()
        except raised:
            failed.append(pin)
    assert failed, f"no pin noticed {name}: {planted!r}"


def test_pins_pass_on_the_oracle_as_written():
    """The same pins, without any edit, pass (the cases above fail them only through the
    planted line)."""
    seen = set()
    for case in CASES:
        for pin in case[5]:
            key = getattr(pin, "__code__", pin)
            if key in seen:
                continue
            seen.add(key)
            pin()
    assert oracle.gmres_right is GM.gmres_right
