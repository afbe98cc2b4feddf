"""Each plausible mistake planted in the oracle (on the CPU) fails a pin.

The oracle source is copied with one textual change, compiled to a temporary
library, and run through every pin of tests/pins.py; at least one pin must
reject it.  This shows the pins constrain every part of the oracle: the
harmonic recurrences, the symmetry, the solid layout, P2M/P2L, evaluation and
the three translations (dropped terms, wrong signs or indices, transposed
operands, single- instead of double-height sums)."""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sfmm_oracle.c")

MUTANTS = {
    "m2l_no_conj": ("s += conj(Mf[hidx(k, l)]) * S[hidx(n + k, m + l)];",
                    "s += Mf[hidx(k, l)] * S[hidx(n + k, m + l)];"),
    "m2l_no_sign": ("s *= sgn(n);", "s *= 1.0;"),
    "m2l_index_m_minus_l": ("s += conj(Mf[hidx(k, l)]) * S[hidx(n + k, m + l)];",
                            "s += conj(Mf[hidx(k, l)]) * S[hidx(n + k, m - l)];"),
    "m2l_drop_l_eq_minus_k": ("for (int l = -k; l <= k; ++l)\n                    s += conj",
                              "for (int l = -k + 1; l <= k; ++l)\n                    s += conj"),
    "m2l_single_height": ("for (int k = 0; k < p_in; ++k)\n                for (int l = -k; l <= k; ++l)\n                    s += conj",
                          "for (int k = 0; k < p_in - n; ++k)\n                for (int l = -k; l <= k; ++l)\n                    s += conj"),
    "R_column_coeff": ("v = ((2.0 * n - 1.0) * z * R[hidx(n - 1, m)] - r2 * rm2)",
                       "v = ((2.0 * n + 1.0) * z * R[hidx(n - 1, m)] - r2 * rm2)"),
    "R_column_drop_term": ("v = ((2.0 * n - 1.0) * z * R[hidx(n - 1, m)] - r2 * rm2)",
                           "v = ((2.0 * n - 1.0) * z * R[hidx(n - 1, m)])"),
    "R_diagonal": ("v = w / (2.0 * n) * R[hidx(n - 1, n - 1)];",
                   "v = w / (1.0 * n) * R[hidx(n - 1, n - 1)];"),
    "S_diagonal": ("v = (2.0 * n - 1.0) * w / r2 * S[hidx(n - 1, n - 1)];",
                   "v = (2.0 * n + 1.0) * w / r2 * S[hidx(n - 1, n - 1)];"),
    "S_column_coeff": ("- ((double)(n - 1) * (n - 1) - (double)m * m) * sm2) / r2;",
                       "- ((double)n * n - (double)m * m) * sm2) / r2;"),
    "S_diag_conj": ("v = (2.0 * n - 1.0) * w / r2 * S[hidx(n - 1, n - 1)];",
                    "v = (2.0 * n - 1.0) * conj(w) / r2 * S[hidx(n - 1, n - 1)];"),
    "symmetry_sign": ("if (R) R[hidx(n, -m)] = sgn(m) * conj(R[hidx(n, m)]);",
                      "if (R) R[hidx(n, -m)] = conj(R[hidx(n, m)]);"),
    "solid_symmetry_sign": ("F[hidx(n, -m)] = sgn(m) * conj(v);", "F[hidx(n, -m)] = conj(v);"),
    "layout_im_offset": ("static int pos_im(int n, int m) { return n * (n + 1) + n + 1 + m; }",
                         "static int pos_im(int n, int m) { return n * (n + 1) + n + m; }"),
    "m2m_shift_sign": ("const double mr[3] = {-r[0], -r[1], -r[2]};",
                       "const double mr[3] = {r[0], r[1], r[2]};"),
    "m2m_transposed_order": ("s += Mf[hidx(k, l)] * R[hidx(n - k, m - l)];",
                             "s += Mf[hidx(k, l)] * R[hidx(n - k, l - m)];"),
    "l2l_no_conj": ("s += Lf[hidx(k, l)] * conj(R[hidx(k - n, l - m)]);",
                    "s += Lf[hidx(k, l)] * R[hidx(k - n, l - m)];"),
    "l2l_transposed_order": ("s += Lf[hidx(k, l)] * conj(R[hidx(k - n, l - m)]);",
                             "s += Lf[hidx(k, l)] * conj(R[hidx(k - n, m - l)]);"),
    "p2m_reversed": ("double d[3] = {pos[3 * j] - centre[0], pos[3 * j + 1] - centre[1],\n                       pos[3 * j + 2] - centre[2]};\n        harmonics(P, d, R, NULL);",
                     "double d[3] = {centre[0] - pos[3 * j], centre[1] - pos[3 * j + 1],\n                       centre[2] - pos[3 * j + 2]};\n        harmonics(P, d, R, NULL);"),
    "p2l_conj": ("for (int i = 0; i < P * P; ++i) acc[i] += q[j] * S[i];",
                 "for (int i = 0; i < P * P; ++i) acc[i] += q[j] * conj(S[i]);"),
    "eval_m_no_conj": ("s += Mf[hidx(n, m)] * conj(S[hidx(n, m)]);",
                       "s += Mf[hidx(n, m)] * S[hidx(n, m)];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(msrc),
                    "-o", str(lib), "-lm"], check=True)
    o = oracle.Oracle(str(lib))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            err, tol = pin(o)
            if not (err <= tol):
                caught.append(pin.__name__)
        except Exception as e:  # an exception also rejects the mutant
            caught.append(pin.__name__ + ":" + type(e).__name__)
    assert caught, f"mutant {name} passed every pin"
