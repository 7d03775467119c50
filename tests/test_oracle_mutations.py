"""Plant plausible mistakes in a copy of the oracle and check that the pins catch every one (CPU only).

Each mutation is a one-line change of ``oracle/bed_oracle.c`` of the kind a transcription error would
make (a dropped term, a wrong sign or index, a transposed operand). The mutated copy is compiled into a
temporary directory and the pin suite ``tests/test_oracle_pins.py`` is run against it in a subprocess;
the suite must fail. All mutations keep every memory access in bounds.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bed_oracle.c")

MUTATIONS = {
    "tear_sign": ("d1[m - 1] -= *rho;", "d1[m - 1] += *rho;"),
    "z_drops_sigma": ("z[j] = sigma * Q1[(m - 1) * m + j];", "z[j] = Q1[(m - 1) * m + j];"),
    "z_first_row_of_Q1": ("z[j] = sigma * Q1[(m - 1) * m + j];", "z[j] = sigma * Q1[j];"),
    "merge_Q1_transposed": ("acc += Q1[r * m + k] * Uq[k * s + c];", "acc += Q1[k * m + r] * Uq[k * s + c];"),
    "secular_drops_a_term": ("        s0 += t;\n", "        s0 += (j == K - 1) ? 0.0 : t;\n"),
    "secular_f2_factor": ("*f2 = 2.0 * rho * s2;", "*f2 = rho * s2;"),
    "secular_sign_of_shift": ("double dl = (d[j] - d[o]) - tau;", "double dl = (d[j] - d[o]) + tau;"),
    "origin_not_moved": ("        o = i - 1;\n        L -= shift;", "        o = i;\n        L -= shift;"),
    "bracket_from_wrong_pole": ("double U = (i == 0) ? (upper0 - d[0]) : (d[i - 1] - d[i]);",
                                "double U = (i == 0) ? (upper0 - d[0]) : (d[0] - d[i]);"),
    "section_update_swapped": ("        it++;\n        ns++;\n        if (f > 0)\n            U = h;\n        else if (f < 0)\n            L = h;",
                               "        it++;\n        ns++;\n        if (f < 0)\n            U = h;\n        else if (f > 0)\n            L = h;"),
    "zhat_sign_dropped": ("zhat[i] = (z[i] >= 0 ? 1.0 : -1.0) * sqrt(q > 0 ? q : 0.0);", "zhat[i] = sqrt(q > 0 ? q : 0.0);"),
    "zhat_ratio_index": ("for (int j = 0; j < i; j++) q *= ((d[origin[j + 1]] - d[i]) + tau[j + 1]) / (d[j] - d[i]);",
                         "for (int j = 0; j < i; j++) q *= ((d[origin[j]] - d[i]) + tau[j]) / (d[j] - d[i]);"),
    "zhat_drops_rho": ("double q = ((d[origin[0]] - d[i]) + tau[0]) / rho;", "double q = ((d[origin[0]] - d[i]) + tau[0]);"),
    "vector_shift_sign": ("double q = zh[i] / ((dK[i] - dK[orig[j]]) - tau[j]);", "double q = zh[i] / ((dK[i] - dK[orig[j]]) + tau[j]);"),
    "rotation_undo_sign": ("Y[q * s + k] = -sn * yp + c * yq;", "Y[q * s + k] = sn * yp + c * yq;"),
    "rotation_new_pole": ("dd[p] = sn * sn * a + c * c * b;", "dd[p] = c * c * a + sn * sn * b;"),
    "householder_tau_sign": ("tau = (beta - alpha) / beta;", "tau = (alpha - beta) / beta;"),
    "householder_w_factor": ("w[i] = p[i] - 0.5 * tau * pv * v[i];", "w[i] = p[i] - tau * pv * v[i];"),
    "backtransform_transposed": ("acc += H[r * n + k] * QT[k * n + c];", "acc += H[k * n + r] * QT[k * n + c];"),
    "leaf_rotation_sign": ("    Q[2] = -sn;\n", "    Q[2] = sn;\n"),
    "sign_convention_flipped": ("if (V[im * n + c] < 0)", "if (V[im * n + c] > 0)"),
    "backward_gap_sign": ("m = vg / (W[j] - W[i]);", "m = vg / (W[i] - W[j]);"),
    "backward_not_symmetrized": ("gA[i * n + j] = 0.5 * (G[i * n + j] + G[j * n + i]);", "gA[i * n + j] = G[i * n + j];"),
    "deflation_drops_rho": ("defl[p] = (rho * fabs(zz[p]) * nz <= tol);", "defl[p] = (fabs(zz[p]) <= 0.5);"),
    "ql_rotation_sign": ("Q[k * s + i + 1] = sn * qa + cs * qb;", "Q[k * s + i + 1] = -sn * qa + cs * qb;"),
    "ql_bulge_term": ("r = (d[i] - g) * sn + 2.0 * cs * b;", "r = (d[i] - g) * sn + cs * b;"),
}


def _run_mutant(name, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name}: pattern must occur exactly once"
    path = os.path.join(workdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(workdir, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", so, path, "-lm", "-lpthread"])
    env = dict(os.environ, BED_ORACLE_LIB=so)
    r = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q", "-p", "no:cacheprovider"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600,
    )
    return r.returncode, r.stdout[-400:]


def test_unmutated_copy_passes_the_pins():
    with tempfile.TemporaryDirectory() as td:
        rc, out = _run_mutant("identity", "#define ORC_U 0x1p-53", "#define ORC_U 0x1p-53", td)
    assert rc == 0, out


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as td, cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run_mutant, name, old, new, td) for name, (old, new) in MUTATIONS.items()}
        survivors = [name for name, f in futs.items() if f.result()[0] == 0]
    assert not survivors, f"pins did not catch: {survivors}"
