"""Planted mistakes in the oracle: each must fail one of its pins.

Every case copies ``oracle/cbg_oracle.c``, replaces one exact snippet by a plausible
mistake (a dropped term, a wrong sign or index, a transposed operand, a wrong constant),
compiles the copy with the oracle's own flags and runs the oracle's pin files
(``test_oracle_codec.py``, ``test_oracle_gmres.py``, ``test_oracle_learned.py``) against
it in a child pytest, through ``CBG_ORACLE_LIB``.  A mistake that leaves every pin green
is a gap in the pins.  An unchanged copy built the same way must pass them all, so that a
failure is the planted mistake's and not the harness's.  CPU only; the planted copies
live in a temporary directory and never replace the oracle.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cbg_oracle.c")
PIN_FILES = {k: os.path.join(ROOT, "tests", f"test_oracle_{k}.py")
             for k in ("codec", "gmres", "learned")}
CODEC = {  # mistakes in the codec: test_oracle_codec.py runs first
    "bf16_max_overflows", "bf16_precision", "e4m3_nan_exponent", "e4m3_no_saturation",
    "e4m3_scale_fmax", "f16_decode_bias", "f16_emin", "f16_max_overflows",
    "int_decode_scale", "int_sigma", "int_truncates", "pow2_scale_not_smallest",
    "round_ties_away", "round_truncates", "subnormal_pack_shift"}
LEARNED = {  # mistakes in the network and SPAI parts: test_oracle_learned.py runs first
    "mlp_forward_no_bias", "mlp_forward_no_relu", "mlp_relu_grad", "mlp_w2_transposed",
    "mlp_w3_grad_operand", "spai_gradient_factor", "spai_loss_cross_term",
    "spai_slots_swapped", "spai_statistic_d"}

# (name, what the mistake is, exact snippet of cbg_oracle.c, its replacement)
MUTANTS = [
    ("round_ties_away", "round-to-nearest with ties away from zero instead of to even",
     "if (rem > 0.5 || (rem == 0.5 && fmod(k, 2.0) != 0.0)) k += 1.0;",
     "if (rem >= 0.5) k += 1.0;"),
    ("round_truncates", "the rounding step dropped (truncation)",
     "if (rem > 0.5 || (rem == 0.5 && fmod(k, 2.0) != 0.0)) k += 1.0;",
     "(void)rem;"),
    ("f16_emin", "binary16 minimum exponent off by one (subnormal range)",
     "double r = round_to_format(x, 11, -14);",
     "double r = round_to_format(x, 11, -15);"),
    ("f16_decode_bias", "binary16 decode with exponent bias 16",
     "return s * unpack_format(expf, man, 10, 15, -14);",
     "return s * unpack_format(expf, man, 10, 16, -14);"),
    ("bf16_precision", "bfloat16 rounded to 7 significand bits instead of 8",
     "double r = round_to_format(x, 8, -126);",
     "double r = round_to_format(x, 7, -126);"),
    ("e4m3_no_saturation", "e4m3 overflow not saturated to 448",
     "if (fabs(r) > 448.0) r = copysign(448.0, x);",
     "(void)0;"),
    ("int_sigma", "fixed-point scale sigma = max|v| / (max_int + 1) (Section 4.2)",
     "double sigma = vmax / mx;",
     "double sigma = vmax / (mx + 1.0);"),
    ("int_truncates", "fixed-point code truncated instead of rounded",
     "double q = rint(v[i] * inv);",
     "double q = trunc(v[i] * inv);"),
    ("int_decode_scale", "int16 decode without its scale",
     "case OR_I16: out[i] = (double)((const int16_t*)codes)[i] * scale; break;",
     "case OR_I16: out[i] = (double)((const int16_t*)codes)[i]; break;"),
    ("pow2_scale_not_smallest", "power-of-two scale one binade too large",
     "    if (e < -126) e = -126;                /* keep the scale a normal FP32 number */\n    return e;",
     "    if (e < -126) e = -126;                /* keep the scale a normal FP32 number */\n    return e + 1;"),
    ("spmv_drops_first_entry", "sparse product skips the first nonzero of every row",
     "for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * x[col[p]];",
     "for (int32_t p = rowptr[i] + 1; p < rowptr[i + 1]; p++) s += val[p] * x[col[p]];"),
    ("dot_drops_first_block", "inner product drops its first block of 4096 terms",
     "for (int64_t k = 0; k < nb; k++) s += part[k];",
     "for (int64_t k = 1; k < nb; k++) s += part[k];"),
    ("residual_sign", "cycle-start residual r = A x - b",
     "for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];",
     "for (int64_t i = 0; i < n; i++) r[i] = r[i] - b[i];"),
    ("cgs_sign", "CGS update w += V c",
     "for (int64_t i = 0; i <= j; i++) wt -= V[(size_t)i * (size_t)n + (size_t)t] * c[i];",
     "for (int64_t i = 0; i <= j; i++) wt += V[(size_t)i * (size_t)n + (size_t)t] * c[i];"),
    ("cgs_skips_last_column", "CGS projects out all columns but the newest",
     "for (int64_t i = 0; i <= j; i++) wt -= V[(size_t)i * (size_t)n + (size_t)t] * c[i];",
     "for (int64_t i = 0; i < j; i++) wt -= V[(size_t)i * (size_t)n + (size_t)t] * c[i];"),
    ("mgs_sign", "MGS update w += c_i v_i",
     "for (int64_t t = 0; t < n; t++) w[t] -= vi[t] * c[i];",
     "for (int64_t t = 0; t < n; t++) w[t] += vi[t] * c[i];"),
    ("reorth_overwrites", "re-orthogonalisation coefficients replace h instead of adding to it",
     "for (int64_t i = 0; i <= j; i++) h[i] += u[i];",
     "for (int64_t i = 0; i <= j; i++) h[i] = u[i];"),
    ("hessenberg_subdiag", "h_{j+1,j} taken before the re-orthogonalisation pass",
     "                hn = nrm2(n, w);\n                a->reorths++;",
     "                a->reorths++;"),
    ("givens_sign", "second row of the Givens rotation with the wrong sign",
     "double t1 = -sn[i] * Rc[i] + cs[i] * Rc[i + 1];",
     "double t1 = sn[i] * Rc[i] + cs[i] * Rc[i + 1];"),
    ("givens_swapped", "c and s of the new rotation swapped",
     "else { cs[j] = Rc[j] / rr; sn[j] = Rc[j + 1] / rr; }",
     "else { cs[j] = Rc[j + 1] / rr; sn[j] = Rc[j] / rr; }"),
    ("g_sign", "rotated right-hand side g_{j+1} = s g_j",
     "g[j + 1] = -sn[j] * g[j];",
     "g[j + 1] = sn[j] * g[j];"),
    ("backsolve_transposed", "back-substitution reads R transposed",
     "for (int64_t c = i + 1; c < k; c++) s -= R[i + c * (m + 1)] * y[c];",
     "for (int64_t c = i + 1; c < k; c++) s -= R[c + i * (m + 1)] * y[c];"),
    ("normalise_dropped", "basis vector stored without dividing by its norm",
     "for (int64_t i = 0; i < n; i++) tmp[i] = w[i] * inv;",
     "for (int64_t i = 0; i < n; i++) tmp[i] = w[i];"),
    ("update_skips_precond", "solution update x += V y without M^{-1}",
     "apply_precond(&P, tmp, z);",
     "memcpy(z, tmp, (size_t)n * sizeof(double));"),
    ("jacobi_multiplies", "Jacobi applies D instead of D^{-1}",
     "for (int64_t i = 0; i < n; i++) z[i] = v[i] / P->dinv_src[i];",
     "for (int64_t i = 0; i < n; i++) z[i] = v[i] * P->dinv_src[i];"),
    ("bj4_transposed", "block-Jacobi stores each block inverse transposed",
     "for (int c = 0; c < kb; c++) B[4 * i + c] = aug[i][kb + c];",
     "for (int c = 0; c < kb; c++) B[4 * c + i] = aug[i][kb + c];"),
    ("adapt_skips_rung", "adaptive ladder jumps e4m3 -> f32",
     "if (f == OR_E4M3) return OR_BF16;",
     "if (f == OR_E4M3) return OR_F32;"),
    ("mlp_relu_grad", "backward pass ignores the second ReLU",
     "d2[i] = a2[i] > 0.0 ? s : 0.0;",
     "d2[i] = s;"),
    ("mlp_w2_transposed", "backward pass multiplies by W2 instead of W2^T",
     "for (int o = 0; o < MLP_H; o++) s += W2[o * MLP_H + i] * d2[o];",
     "for (int o = 0; o < MLP_H; o++) s += W2[i * MLP_H + o] * d2[o];"),
    ("spai_loss_cross_term", "SPAI loss cross term without its factor 2",
     "li += pv[k] * gp - 2.0 * pv[k] * c[i * 7 + k];",
     "li += pv[k] * gp - pv[k] * c[i * 7 + k];"),
    ("conditional_reorth_inverted", "conditional re-orthogonalisation when ||w|| >= eta omega",
     "(a->reorth == OR_REORTH_CONDITIONAL && hn < a->eta * omega);",
     "(a->reorth == OR_REORTH_CONDITIONAL && hn >= a->eta * omega);"),
    ("breakdown_unscaled", "breakdown test against eps instead of eps omega",
     "int stop = !(hn > a->eps_bd * omega);",
     "int stop = !(hn > a->eps_bd);"),
    ("omega_of_z", "omega taken from M^{-1} v_j instead of w = A M^{-1} v_j",
     "double omega = nrm2(n, w);",
     "double omega = nrm2(n, z);"),
    ("adapt_condition_inverted", "adaptive switch when the explicit residual is below the gap",
     "if (a->adapt && a->cycles > 0 && beta > a->adapt_gap * last_est) {",
     "if (a->adapt && a->cycles > 0 && beta < a->adapt_gap * last_est) {"),
    ("residual_estimate_index", "recurrence residual read from g_j instead of g_{j+1}",
     "double est = fabs(g[j + 1]);",
     "double est = fabs(g[j]);"),
    ("restart_discards_x", "restart replaces x by the last correction",
     "for (int64_t t = 0; t < n; t++) x[t] += z[t];",
     "for (int64_t t = 0; t < n; t++) x[t] = z[t];"),
    ("f16_max_overflows", "binary16 65504 encoded as infinity",
     "if (fabs(r) > 65504.0) return (uint16_t)(sign | 0x7C00u);",
     "if (fabs(r) >= 65504.0) return (uint16_t)(sign | 0x7C00u);"),
    ("bf16_max_overflows", "bfloat16 largest finite value encoded as infinity",
     "if (fabs(r) > 0x1.FEp127) return (uint16_t)(sign | 0x7F80u);",
     "if (fabs(r) >= 0x1.FEp127) return (uint16_t)(sign | 0x7F80u);"),
    ("e4m3_nan_exponent", "e4m3 decode treats every exponent-15 pattern as NaN (IEEE-style)",
     "if (expf == 0xFu && man == 0x7u) return NAN;",
     "if (expf == 0xFu) return NAN;"),
    ("subnormal_pack_shift", "subnormal mantissa packed one bit low",
     "man = (uint32_t)ldexp(a, mbits - emin);",
     "man = (uint32_t)ldexp(a, mbits - emin - 1);"),
    ("e4m3_scale_fmax", "e4m3 scale chosen for a maximum of 256 instead of 448",
     "int e = pow2_scale_exponent(vmax, fmt == OR_BF16 ? 1.0 : 448.0);",
     "int e = pow2_scale_exponent(vmax, fmt == OR_BF16 ? 1.0 : 256.0);"),
    ("bj4_elimination_sign", "Gauss-Jordan elimination adds the pivot row",
     "for (int c = 0; c < 2 * kb; c++) aug[i][c] = aug[i][c] - f * aug[k][c];",
     "for (int c = 0; c < 2 * kb; c++) aug[i][c] = aug[i][c] + f * aug[k][c];"),
    ("mlp_forward_no_bias", "network forward drops the first layer's bias",
     "double s = b1[o];",
     "double s = 0.0;"),
    ("mlp_forward_no_relu", "network forward without the first ReLU",
     "a1[o] = s > 0.0 ? s : 0.0;",
     "a1[o] = s;"),
    ("mlp_w3_grad_operand", "W3 gradient multiplies by the first hidden layer",
     "for (int i = 0; i < MLP_H; i++) gW3[o * MLP_H + i] += go[o] * a2[i];",
     "for (int i = 0; i < MLP_H; i++) gW3[o * MLP_H + i] += go[o] * a1[i];"),
    ("spai_slots_swapped", "stencil slots of the -x and -y neighbours swapped",
     "const int64_t off[7] = {-sxy, -sx, -1, 0, 1, sx, sxy};",
     "const int64_t off[7] = {-sx, -sxy, -1, 0, 1, sx, sxy};"),
    ("spai_statistic_d", "pair statistic d without the square of e",
     "d[i] += wgt * e[i] * e[i];",
     "d[i] += wgt * e[i];"),
    ("spai_gradient_factor", "SPAI loss gradient without its factor 2",
     "if (gout) gout[i * 7 + k] = has[k] ? 2.0 * (gp - c[i * 7 + k]) / diag[i] / npairs : 0.0;",
     "if (gout) gout[i * 7 + k] = has[k] ? (gp - c[i * 7 + k]) / diag[i] / npairs : 0.0;"),
]


def _cflags():
    sys.path.insert(0, ROOT)
    import oracle
    return list(oracle.CFLAGS)


def _build(src_text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    inc = os.path.join(ROOT, "oracle")
    subprocess.check_call(["gcc"] + _cflags() + ["-I", inc, "-o", path, c, "-lm"])
    return path


def _region(name):
    return "codec" if name in CODEC else "learned" if name in LEARNED else "gmres"


def _run_pins(lib_path, first):
    """Exit status of the pin files against the library: the file of the mistake's own
    region first, the other two only if it passes (0: every pin passed, 1: one failed)."""
    env = dict(os.environ, CBG_ORACLE_LIB=lib_path, OMP_NUM_THREADS="2")
    rest = [f for k, f in PIN_FILES.items() if k != first]
    out = ""
    for files in ([PIN_FILES[first]], rest):
        p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"] + files,
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        out += p.stdout[-1500:]
        if p.returncode != 0:
            return p.returncode, out
    return 0, out


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(SRC).read()
    d = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = {"control": src}
    assert CODEC | LEARNED <= {m[0] for m in MUTANTS}
    for name, _, old, new in MUTANTS:
        assert src.count(old) == 1, f"{name}: snippet not found exactly once in cbg_oracle.c"
        jobs[name] = src.replace(old, new)

    def one(item):
        name, text = item
        return name, _run_pins(_build(text, os.path.join(d, f"lib_{name}.so")), _region(name))

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(one, jobs.items()))


def test_unchanged_copy_passes_every_pin(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name,what", [(m[0], m[1]) for m in MUTANTS], ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name, what):
    rc, out = outcomes[name]
    # exit status 1: tests ran and at least one failed (not a crash or a collection error)
    assert rc == 1, f"{name} ({what}) was not caught by any pin (exit {rc}):\n{out}"
