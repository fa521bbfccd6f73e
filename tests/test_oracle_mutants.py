"""The pins catch plausible mistakes in the oracle.  Each case plants one
mistake -- a dropped term, a flipped sign, a transposed operand, the paper's
printed copy error, a wrong axis, a swapped order of operations -- in a copy
of oracle/sdgr_oracle.c, compiles it, and runs tests/test_oracle_pins.py
against that build in a child process: at least one pin must fail.  The
unchanged source, built the same way, passes them all."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sdgr_oracle.c")

MUTANTS = {
    "dilation dropped on the imaging plane": [(
        "g->S2[pl][a][b] = acc + (a == b ? cfg->eps : 0.0);",
        "g->S2[pl][a][b] = acc + (a == b && pl == 0 ? cfg->eps : 0.0);")],
    "transposed rotation in Sigma_r": [(
        "acc += g->Rr[a][i] * g->Sig[i][j] * g->Rr[b][j];",
        "acc += g->Rr[i][a] * g->Sig[i][j] * g->Rr[j][b];")],
    "printed tan(theta) kept in the range row of P_I": [(
        "2.0 / (v->dR * v->NR) * g->xr[2]",
        "2.0 / (v->dR * v->NR * tt) * g->xr[2]")],
    "pixel centres at half-integers": [(
        "g->u[0][k] = (ndcC[k] + 1.0) * Ns[k] * 0.5 - 0.5;",
        "g->u[0][k] = (ndcC[k] + 1.0) * Ns[k] * 0.5;")],
    "attenuation applied before the deposit": [(
        "Ap[i] += alpha * T;\n                T *= (1.0 - alpha);",
        "T *= (1.0 - alpha);\n                Ap[i] += alpha * T;")],
    "normaliser without the square root": [(
        "1.0 / (2.0 * ORC_PI * sqrt(g->det[1]))",
        "1.0 / (2.0 * ORC_PI * g->det[1])")],
    "depth order reversed": [(
        "if (ka < kb) return -1;\n    if (ka > kb) return 1;",
        "if (ka > kb) return -1;\n    if (ka < kb) return 1;")],
    "depth key from the elevation axis": [(
        "g->key = (double)(float)(g->Rr[2][0] * d[0] + g->Rr[2][1] * d[1] + g->Rr[2][2] * d[2]);",
        "g->key = (double)(float)(g->Rr[1][0] * d[0] + g->Rr[1][1] * d[1] + g->Rr[1][2] * d[2]);")],
    "suffix sum without the (1 - alpha) factor": [(
        "B = chat[j] * al[k] + (1.0 - al[k]) * B;",
        "B = chat[j] * al[k] + B;")],
    "conic adjoint with the wrong sign": [(
        "acc[3] += gE * (-0.5 * e1 * d[0] * d[0]);",
        "acc[3] += gE * (0.5 * e1 * d[0] * d[0]);")],
    "dL/dP with I instead of A": [(
        "gr[7] += ad->gI * A[i];",
        "gr[7] += ad->gI * A[i] * q->P;")],
    "opacity chain rule without (1 - o)": [(
        "gr[3] += ad->o * (cfg->alpha_mode ? q->o : q->o * (1.0 - q->o));",
        "gr[3] += ad->o * q->o;")],
    "Adam without the first-moment bias correction": [(
        "double mh = m[i] / bc1, vh = v[i] / bc2;",
        "double mh = m[i], vh = v[i] / bc2;")],
    "L1 gradient with the wrong sign": [(
        "dLdS[k] = (r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0)) / (double)npix;",
        "dLdS[k] = (r > 0.0 ? -1.0 : (r < 0.0 ? 1.0 : 0.0)) / (double)npix;")],
    "SH degree-1 basis with y and x swapped": [(
        "Y[0] = c1 * y; Y[1] = c1 * z; Y[2] = c1 * x;",
        "Y[0] = c1 * x; Y[1] = c1 * z; Y[2] = c1 * y;")],
}


def _build(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) >= 1, (name, old)
        src = src.replace(old, new, 1)
    c = tmp_path / ("m%d.c" % abs(hash(name)))
    c.write_text(src)
    so = tmp_path / ("m%d.so" % abs(hash(name)))
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"])
    return str(so)


def _pins(lib_path):
    env = dict(os.environ, SDGR_ORACLE_LIB=lib_path, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join("tests", "test_oracle_pins.py")], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return p.returncode, p.stdout[-1500:]


def test_unchanged_source_passes(tmp_path):
    code, out = _pins(_build(tmp_path, "unchanged", []))
    assert code == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    code, out = _pins(_build(tmp_path, name, MUTANTS[name]))
    assert code != 0, "no pin failed for: " + name
    assert "failed" in out, out
