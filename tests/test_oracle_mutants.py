"""Mutation check of the oracle's pins: plant a plausible mistake in a temporary copy of the
oracle's C source, rebuild it, and require that the pin aimed at that mistake fails.

Nothing is changed in ``oracle/``; each mutant lives in a pytest tmp directory.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import tests.test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sfseg_oracle.c")

# (name, text in the oracle, planted replacement, pins that must fail)
MUTANTS = [
    ("eq7_third_term_sign", "+ 2.0 * u[i] * f[i] * c3[i]", "- 2.0 * u[i] * f[i] * c3[i]",
     ["test_kronecker_closed_form"]),
    ("eq7_dropped_f2_term", "- u[i] * c2[i]", "- 0.0 * c2[i]",
     ["test_kronecker_closed_form"]),
    ("eq2_pair_sign", "(1.0 - alpha * df * df)", "(1.0 + alpha * df * df)",
     ["test_two_node_closed_form"]),
    ("filter_axes_swapped", "filter_axis(T, H, W, 2, rw, gw, in, out);",
     "filter_axis(T, H, W, 2, rh, gh, in, out);", ["test_kronecker_closed_form"]),
    ("unary_exponent", "return s > 0.0 ? pow(s, p) : 0.0;", "return s > 0.0 ? pow(s, 2.0 * p) : 0.0;",
     ["test_diagonal_special_case"]),
    ("sigmoid_sign", "f[i] = 1.0 / (1.0 + exp(-z));", "f[i] = 1.0 / (1.0 + exp(z));",
     ["test_combine_sigmoid_is_logistic"]),
    ("gradient_pair_sign", "- 2.0 * alpha * ua * ub * d;", "+ 2.0 * alpha * ua * ub * d;",
     ["test_grad_matches_finite_differences"]),
    ("edge_padding_off_by_one", "int lo = pos - r < 0 ? -pos : -r;",
     "int lo = pos - r < 0 ? 1 - pos : -r;",
     ["test_filter_form_equals_explicit_matrix"]),
    ("l1_renormalisation",
     "orc_spmv(N, rowptr, col, val, x_out, y);\n        double nu = sqrt(orc_sumsq(y, N));",
     "orc_spmv(N, rowptr, col, val, x_out, y);\n        double nu = 0.0;\n"
     "        for (int64_t q = 0; q < N; ++q) nu += fabs(y[q]);",
     ["test_two_node_closed_form", "test_power_iteration_matches_dense_eigensolver"]),
    ("eq1_pair_not_squared", "exp(-alpha * df * df)", "exp(-alpha * fabs(df))",
     ["test_exact_kernel_kronecker_closed_form"]),
    ("eq1_pair_sign", "exp(-alpha * df * df)", "exp(alpha * df * df)",
     ["test_exact_kernel_kronecker_closed_form", "test_exact_kernel_approaches_taylor"]),
    ("binarize_no_max_scaling", "exp(-gain * (y[i] / m - center))", "exp(-gain * (y[i] - center))",
     ["test_soft_binarize_kronecker_closed_form"]),
    ("binarize_sigmoid_sign", "exp(-gain * (y[i] / m - center))", "exp(gain * (y[i] / m - center))",
     ["test_soft_binarize_kronecker_closed_form"]),
    ("binarize_operator_skipped",
     "orc_filter_apply(T, H, W, s, f, p, alpha, rt, rh, rw, st, sh, sw, x_out, y);\n        double m = y[0];",
     "for (int64_t q = 0; q < N; ++q) y[q] = x_out[q];\n        double m = y[0];",
     ["test_soft_binarize_diagonal_two_steps"]),
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           str(path), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    for name, rt in [("orc_build_affinity", ctypes.c_int64), ("orc_sumsq", ctypes.c_double),
                     ("orc_dot", ctypes.c_double), ("orc_power_csr", ctypes.c_int),
                     ("orc_power_filter", ctypes.c_int), ("orc_grad_csr", ctypes.c_int),
                     ("orc_num_threads", ctypes.c_int)]:
        getattr(lib, name).restype = rt
    return lib


def _run_pin(name):
    fn = getattr(pins, name)
    if name == "test_grad_matches_finite_differences":
        fn("linear")
    elif name == "test_filter_form_equals_explicit_matrix":
        fn((3, 5, 7), (1, 2, 2), None, 1.0, 0.1)
    else:
        fn()


@pytest.mark.parametrize("name,old,new,targets", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, monkeypatch, name, old, new, targets):
    lib = _build_mutant(tmp_path, old, new)
    oracle._load()                      # make sure the real library is loaded first
    monkeypatch.setattr(oracle, "_lib", lib)
    for t in targets:
        with pytest.raises((AssertionError, FloatingPointError)):
            _run_pin(t)


# Mistakes planted in the Python-level oracle functions (a modified copy of the function's source
# is executed in the oracle's namespace and patched in for the duration of the test).
PY_MUTANTS = [
    ("online_new_frame_uniform", "online",
     "newest = xw[-1] if k > 0 else np.ones((H, W))", "newest = np.ones((H, W))",
     ["test_online_diagonal_closed_form"]),
    ("online_shift_backwards", "online",
     "xw = np.concatenate([xw[1:], newest[None]])", "xw = np.concatenate([newest[None], xw[:-1]])",
     ["test_online_diagonal_closed_form", "test_online_start_vectors"]),
]


@pytest.mark.parametrize("name,func,old,new,targets", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pin_catches_planted_python_mistake(monkeypatch, name, func, old, new, targets):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(oracle, func)))
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    monkeypatch.setattr(oracle, func, ns[func])
    for t in targets:
        with pytest.raises((AssertionError, FloatingPointError)):
            getattr(pins, t)()
