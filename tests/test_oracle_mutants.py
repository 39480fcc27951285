"""Planted mistakes in the oracle, on the CPU: the pins must catch each one.

Every mutant is a copy of one oracle source with a single plausible error of the
kind a restatement of the paper can carry (a dropped term, a flipped sign, an
operand transposed, an index off by one, a wrong constant).  C mutants of
``oracle/tdc_oracle.c`` are compiled to a scratch library and bound in a child
process (a planted mistake may crash; the child keeps that away from the test
run); numpy mutants of ``oracle/adjoint.py`` and ``oracle/srrsc.py`` are
executed into a fresh module.  The pin tests of ``test_oracle_pins.py``,
``test_oracle_adjoint.py`` and ``test_oracle_srrsc.py`` then run against the
mutant, and at least one of them must fail.  A mutant that survives is a pin
that is missing.  Mutants that change nothing observable (another valid tree
split, a different but convergent shift) are not listed.
"""
import importlib.util
import json
import os
import subprocess
import sys
import types
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")

# (name, fragment of tdc_oracle.c, replacement, what the mistake is)
C_MUTANTS = [
    ("corner_sign", "d[mid] -= fabs(b);", "d[mid] += fabs(b);",
     "Eq. (T2): corner modification of the second child with the wrong sign"),
    ("corner_dropped", "d[mid - 1] -= fabs(b);", ";",
     "Eq. (T2): corner modification of the first child dropped"),
    ("rho_factor", "double rho = 2.0 * fabs(b);", "double rho = fabs(b);",
     "Eq. (T3): rho without the factor 2 of ||v||^2"),
    ("z_scale_dropped", "for (int i = n1; i < n; ++i) z[i] = sg * Q[n1 + (int64_t)i * ldq] * rs2;",
     "for (int i = n1; i < n; ++i) z[i] = sg * Q[n1 + (int64_t)i * ldq];",
     "Eq. (T3): 1/sqrt(2) dropped from the second half of z"),
    ("z_sign_of_b", "double sg = b < 0.0 ? -1.0 : 1.0;", "double sg = 1.0;",
     "Eq. (T2): sign of the coupling entry not folded into z"),
    ("z_row_off_by_one", "z[i] = Q[(n1 - 1) + (int64_t)i * ldq] * rs2;", "z[i] = Q[n1 + (int64_t)i * ldq] * rs2;",
     "Eq. (T3): first half of z taken from the wrong row of diag(Q1, Q2)"),
    ("secular_tau_sign", "double del = (D[i] - D[org]) - tau;", "double del = (D[i] - D[org]) + tau;",
     "Eq. (d-lambda): root offset added instead of subtracted in f"),
    ("secular_origin", "if (g >= 0.0) { org = j; lo = 0.0; hi = 0.5 * gap; }",
     "if (g < 0.0) { org = j; lo = 0.0; hi = 0.5 * gap; }",
     "secular equation: origin taken at the farther pole"),
    ("secular_last_bracket", "org = K - 1; lo = 0.0; hi = rho * zz;", "org = K - 1; lo = 0.0; hi = zz;",
     "secular equation: bracket of the largest root without rho"),
    ("lowner_rho", "double p = ((D[org[K - 1]] - D[i]) + tau[K - 1]) / rho;",
     "double p = ((D[org[K - 1]] - D[i]) + tau[K - 1]) * rho;",
     "Loewner formula: rho multiplies instead of divides"),
    ("lowner_sign", "zhat[i] = copysign(sqrt(p), z[i]);", "zhat[i] = sqrt(p);",
     "Loewner formula: the sign of z_i dropped"),
    ("lowner_pole_shift", "for (int j = 0; j < i; ++j) p *= ((D[org[j]] - D[i]) + tau[j]) / (D[j] - D[i]);",
     "for (int j = 0; j < i; ++j) p *= ((D[org[j]] - D[i]) + tau[j]) / (D[j + 1] - D[i]);",
     "Loewner formula: the poles below i paired with the wrong root"),
    ("colnorm_sqrt", "s[j] = 1.0 / sqrt(acc);", "s[j] = 1.0 / acc;",
     "Eq. (eigenvector): column normaliser without the square root"),
    ("colnorm_tau_sign", "double del = (D[i] - D[org[j]]) - tau[j];\n      double t = zhat[i] / del;",
     "double del = (D[i] - D[org[j]]) + tau[j];\n      double t = zhat[i] / del;",
     "Eq. (d-lambda): root offset with the wrong sign in the normaliser"),
    ("qhat_transposed", "U[i + (int64_t)j * ldu] = zhat[i] * s[j] / del;",
     "U[i + (int64_t)j * ldu] = zhat[j] * s[i] / del;",
     "Eq. (Q_Cauchy): generators of Qhat transposed"),
    ("merge_qhat_transposed", "double u = zh[i] * sn[j] / del;", "double u = zh[j] * sn[i] / del;",
     "Eq. (evect): generators transposed in the merge's vector update"),
    ("merge_root_index", "double del = (Dk[i] - Dk[org[j]]) - tau[j];", "double del = (Dk[i] - Dk[j]) - tau[j];",
     "Eq. (d-lambda): the root index used instead of its origin pole"),
    ("merge_eigenvalue", "for (int j = 0; j < K; ++j) val[j] = Dk[org[j]] + tau[j];",
     "for (int j = 0; j < K; ++j) val[j] = Dk[j] + tau[j];",
     "eigenvalue formed from the root index instead of its origin pole"),
    ("merge_unsorted", "lam[p] = val[ord[p]];", "lam[p] = val[p];",
     "eigenvalues not permuted with their vectors"),
    ("deflate_rotation_sign", "qi[r] = -s * a + c * b;", "qi[r] = s * a + c * b;",
     "Section 3.2: type-2 rotation applied to Q with the wrong sign"),
    ("deflate_pole_swap", "D[pj] = dp * c * c + di * s * s;", "D[pj] = dp * s * s + di * c * c;",
     "Section 3.2: the rotated poles exchanged"),
    ("deflate_tolerance", "double tol = 8.0 * ORC_EPS * fmax(dmax, zmax);",
     "double tol = 8.0e6 * ORC_EPS * fmax(dmax, zmax);",
     "Section 3.2: deflation tolerance a million times too loose"),
    ("leaf_rotation_sign", "vk1[i] = -s * a0 + c * a1;", "vk1[i] = s * a0 + c * a1;",
     "leaf QR: Givens rotation accumulated with the wrong sign"),
    ("leaf_dropped_term", "d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;",
     "d[k] = c * c * ak + 2.0 * c * s * bk;",
     "leaf QR: a term of the rotated diagonal dropped"),
    ("leaf_offdiag_sign", "e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;",
     "e[k] = c * s * (ak - ak1) + (c * c - s * s) * bk;",
     "leaf QR: the rotated off-diagonal with the wrong sign"),
    ("leaf_sort_order", "if (d[j] < d[m]) m = j;", "if (d[j] > d[m]) m = j;",
     "leaf QR: eigenvalues sorted descending"),
    ("tree_depth_off_by_one", "while (((n + ((int64_t)1 << t) - 1) >> t) > leaf) ++t;",
     "while (((n + ((int64_t)1 << t) - 1) >> t) >= leaf) ++t;",
     "tree depth one level too deep at exact powers"),
    ("sign_convention", "if (q[im] < 0.0)", "if (q[im] > 0.0)",
     "column sign convention reversed"),
]

# (file, name, fragment, replacement, what the mistake is)
PY_MUTANTS = [
    ("adjoint.py", "sym_not_skew", "S = 0.5 * (W - W.T)", "S = 0.5 * (W + W.T)",
     "F o sym instead of F o skew"),
    ("adjoint.py", "F_sign", "F[i, j] = 1.0 / (lam[j] - lam[i])", "F[i, j] = 1.0 / (lam[i] - lam[j])",
     "eigenvalue gaps with the wrong sign"),
    ("adjoint.py", "offdiag_factor", "e_bar = 2.0 * np.array", "e_bar = 1.0 * np.array",
     "off-diagonal cotangent without the factor 2 of its two entries"),
    ("adjoint.py", "basis_transposed", "Tb = Q @ M @ Q.T", "Tb = Q.T @ M @ Q",
     "cotangent rotated back with the transposed basis"),
    ("adjoint.py", "lam_bar_only", "M = M + np.diag(", "M = np.diag(",
     "eigenvector part dropped when both cotangents are given"),
    ("srrsc.py", "node_offset_sign", "return (self.d[i] - self.wo[j]) - self.wt[j]",
     "return (self.d[i] - self.wo[j]) + self.wt[j]",
     "Eq. (d-lambda): root offset with the wrong sign in d_i - w_j"),
    ("srrsc.py", "theorem1_u_inverted", "u[i] *= nodes.dd(i, pk) / nodes.dw(i, qk)",
     "u[i] *= nodes.dw(i, qk) / nodes.dd(i, pk)",
     "Theorem 1: row generator update inverted"),
    ("srrsc.py", "theorem1_v_sign", "v[j] *= nodes.ww(j, qk) / nodes.wd(j, pk)",
     "v[j] *= -nodes.ww(j, qk) / nodes.wd(j, pk)",
     "Theorem 1: column generator update with the wrong sign"),
    ("srrsc.py", "theorem2_updated_v", "p = nodes.dw(pi, ci) / v0[ci]", "p = nodes.dw(pi, ci) / v[ci]",
     "Theorem 2: y from the updated instead of the original generator"),
    ("srrsc.py", "geneZ_sign", "Z[a, b] = y[a] * v[j] / nodes.ww(piv_cols[a], j)",
     "Z[a, b] = y[a] * v[j] / nodes.ww(j, piv_cols[a])",
     "Eq. (geneZ): node difference with the wrong sign"),
]


# semi-pinned rank pattern of Table 2: seconds of pure-Python pivoting per run and no
# exact value to compare, so it is left out of the battery
SKIP = ("test_table2_rank_pattern_semi_pinned",)


def battery(module, orc):
    """Run every test function of a pin module (all parametrisations); return the
    names of those that failed or raised."""
    failed = []
    for name in sorted(dir(module)):
        fn = getattr(module, name)
        if not (name.startswith("test_") and callable(fn)) or name in SKIP:
            continue
        cases = [dict()]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name == "parametrize":
                names = [s.strip() for s in mark.args[0].split(",")]
                cases = [dict(c, **dict(zip(names, v if len(names) > 1 else (v,))))
                         for c in cases for v in mark.args[1]]
        params = fn.__code__.co_varnames[:fn.__code__.co_argcount]
        for c in cases:
            kw = dict(c)
            if "orc" in params:
                kw["orc"] = orc
            try:
                with np.errstate(all="ignore"):
                    fn(**kw)
            except Exception as ex:  # AssertionError, LinAlgError, RuntimeError ...
                failed.append("%s%s: %s" % (name, sorted(c.values()) if c else "", type(ex).__name__))
    return failed


def load_test_module(name):
    spec = importlib.util.spec_from_file_location("mut_" + name, os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


_CHILD = r"""
import ctypes, json, os, sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(here)r)
import oracle
oracle._lib = oracle._bind(ctypes.CDLL(sys.argv[1]))
import test_oracle_mutants as tm
pins = tm.load_test_module("test_oracle_pins")
adj = tm.load_test_module("test_oracle_adjoint")
print("FAILED " + json.dumps(tm.battery(pins, oracle) + tm.battery(adj, oracle)))
"""


def _compile(src, out):
    subprocess.check_call(["gcc", "-O1", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=c99", "-o", out, src, "-lm"])


def _run_c_mutant(tmp, name, text):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as f:
        f.write(text)
    _compile(src, lib)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = _CHILD % {"root": ROOT, "here": HERE}
    try:
        p = subprocess.run([sys.executable, "-c", code, lib], capture_output=True, text=True, timeout=300, env=env)
    except subprocess.TimeoutExpired:
        return ["timeout"]
    if p.returncode != 0:
        return ["child exited with %d" % p.returncode]
    line = [l for l in p.stdout.splitlines() if l.startswith("FAILED ")]
    return json.loads(line[-1][7:]) if line else ["no report"]


def test_c_fragments_are_unique():
    src = open(os.path.join(ORACLE, "tdc_oracle.c")).read()
    for name, old, new, _ in C_MUTANTS:
        assert src.count(old) == 1, name
        assert old != new


def test_unmutated_oracle_passes_the_battery(tmp_path):
    # the harness itself: the oracle as it stands, compiled the same way, fails nothing
    src = open(os.path.join(ORACLE, "tdc_oracle.c")).read()
    assert _run_c_mutant(str(tmp_path), "unmutated", src) == []


def test_every_c_mutant_is_caught(tmp_path):
    src = open(os.path.join(ORACLE, "tdc_oracle.c")).read()
    jobs = [(name, src.replace(old, new)) for name, old, new, _ in C_MUTANTS]
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda j: (j[0], _run_c_mutant(str(tmp_path), *j)), jobs))
    survivors = [name for name, failed in results if not failed]
    assert not survivors, "mutants not caught by any pin: %s" % survivors


@pytest.mark.parametrize("fname,name,old,new,why", PY_MUTANTS, ids=[m[1] for m in PY_MUTANTS])
def test_numpy_mutant_is_caught(orc, fname, name, old, new, why):
    path = os.path.join(ORACLE, fname)
    text = open(path).read()
    assert text.count(old) == 1
    mut = types.ModuleType("mutant_" + name)
    exec(compile(text.replace(old, new), path + ":" + name, "exec"), mut.__dict__)
    if fname == "adjoint.py":
        tmod = load_test_module("test_oracle_adjoint")
        tmod.adjoint = mut.adjoint
    else:
        tmod = load_test_module("test_oracle_srrsc")
        for sym in ("Nodes", "dense_block", "reconstruct", "srrsc"):
            setattr(tmod, sym, getattr(mut, sym))
    assert battery(tmod, orc), "planted mistake %s (%s) not caught" % (name, why)
