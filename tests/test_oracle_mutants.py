"""Plant one plausible mistake at a time in a copy of the oracle (on the CPU)
and require that at least one pin catches it. This is evidence that the pins
constrain every part of the oracle, not a test of the oracle itself."""

import os
import shutil
import subprocess

import pytest

import oracle
from oracle import build as obuild
from tests import pins

# (name, original text, planted mistake)
MUTANTS = [
    ("bicgstab_p_sign", "p[i] = r[i] + beta * (p[i] - omega * v[i]);",
     "p[i] = r[i] + beta * (p[i] + omega * v[i]);"),
    ("bicgstab_drop_omega_x", "x[i] = x[i] + alpha * ph[i] + omega * sh[i];",
     "x[i] = x[i] + alpha * ph[i];"),
    ("bicgstab_sigma_shadow", "const double sigma = dot(rh, v, n);",
     "const double sigma = dot(r, v, n);"),
    ("bicgstab_beta_term", "(rho / rho_old) * (alpha / omega)", "(rho / rho_old)"),
    ("bicgstab_omega_swap", "omega = (tt == 0.0) ? 0.0 : ts / tt;",
     "omega = (tt == 0.0) ? 0.0 : tt / ts;"),
    ("spmv_dense_transposed", "sum = sum + A->vals[(size_t)i * n + j] * x[j];",
     "sum = sum + A->vals[(size_t)j * n + i] * x[j];"),
    ("spmv_ell_row_major", "sum = sum + A->vals[(size_t)j * n + i] * x[c];",
     "sum = sum + A->vals[(size_t)i * A->ell_k + j] * x[c];"),
    ("spmv_csr_row_index", "sum = sum + A->vals[e] * x[A->col_idxs[e]];",
     "sum = sum + A->vals[e] * x[i];"),
    ("cg_ratio_inverted", "const double ratio = rho_hat / rho;",
     "const double ratio = rho / rho_hat;"),
    ("cg_r_update_operand", "r[i] = r[i] - alpha * t[i];", "r[i] = r[i] - alpha * p[i];"),
    ("gmres_givens_sign", "H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;",
     "H[(i + 1) * m + j] = sn[i] * a + cs[i] * c;"),
    ("gmres_backsub_sign", "sum = sum - H[i * m + l] * y[l];", "sum = sum + H[i * m + l] * y[l];"),
    ("gmres_update_no_precond", "x[l] = x[l] + u[l];", "x[l] = x[l] + zz[l];"),
    ("ilu_no_pivot_division", "lu[e] = lu[e] / pivot;", "lu[e] = lu[e];"),
    ("ilu_update_sign", "lu[g] = lu[g] - lu[e] * lu[f];", "lu[g] = lu[g] + lu[e] * lu[f];"),
    ("ilu_forward_uses_upper", "            if (ci[e] < i)\n                sum = sum - lu[e] * z[ci[e]];",
     "            if (ci[e] > i)\n                sum = sum - lu[e] * z[ci[e]];"),
    ("ilu_backward_no_diagonal", "z[i] = sum / (d != 0.0 ? d : 1.0);", "z[i] = sum;"),
    ("gmres_mgs_index", "const double *vi = V + (size_t)i * n;", "const double *vi = V + (size_t)j * n;"),
    ("jacobi_not_inverted", "dinv[i] = (precond == OM_JACOBI && d != 0.0) ? 1.0 / d : 1.0;",
     "dinv[i] = (precond == OM_JACOBI && d != 0.0) ? d : 1.0;"),
    ("dot_short", "for (int i = 0; i < n; ++i)\n        sum = sum + a[i] * b[i];\n    return sum;\n}\n\nstatic float",
     "for (int i = 0; i < n - 1; ++i)\n        sum = sum + a[i] * b[i];\n    return sum;\n}\n\nstatic float"),
    ("residual_sign", "r[i] = b[i] - tmp[i];", "r[i] = tmp[i] - b[i];"),
    ("relative_tol_scale", "? o->tol * nb : o->tol", "? o->tol * nb * 100.0 : o->tol"),
    ("refine_no_scale", "x[i] = x[i] + rn * (double)d[i];", "x[i] = x[i] + (double)d[i];"),
    ("refine_inner_shadow", "const float sigma = dot32(rh, v, n);", "const float sigma = dot32(r, v, n);"),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def _build_mutant(workdir, name, before, after):
    src = open(obuild.SRC).read()
    assert src.count(before) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(before, after, 1)
    path = os.path.join(workdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(mutated)
    lib = os.path.join(workdir, f"lib{name}.so")
    subprocess.run([shutil.which("gcc") or "gcc", *obuild.CFLAGS, path, "-o", lib, "-lm"],
                   check=True)
    return lib


@pytest.mark.parametrize("name,before,after", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(workdir, name, before, after):
    lib = _build_mutant(workdir, name, before, after)
    caught = []
    with oracle.using(lib):
        for check in pins.ALL_CHECKS:
            try:
                fails = check()
            except Exception as e:  # a crash or non-finite result also counts as caught
                fails = [f"{type(e).__name__}: {e}"]
            if fails:
                caught.append(check.__name__)
                break
    assert caught, f"no pin caught mutant {name}"
