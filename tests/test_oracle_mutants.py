"""The pins catch planted slips in the oracle.

Each case copies the oracle, plants one plausible mistake in its C source (or
in the selection and OR that its Python wrapper composes) and runs the pins of
that part against the copy (on the CPU); the pins must fail.  Sign flips of the
symmetric taps are not mistakes in effect and are not planted.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "taps_not_normalised": ("for (int o = -R; o <= R; ++o) g[o + R] /= sum;", ""),
    "radius_floor": ("return (int)ceil(truncation * sigma);",
                     "return (int)floor(truncation * sigma);"),
    "z_pass_shifted": ("t2[(i * ey + j) * ezh + (k + rz + o)]",
                       "t2[(i * ey + j) * ezh + (k + rz + o + 1 < ezh ? k + rz + o + 1 : k + rz + o)]"),
    "x_pass_on_y_axis": ("at(d, nx, ny, nz, x + o, y, z, take_abs)",
                         "at(d, nx, ny, nz, x, y + o, z, take_abs)"),
    "edge_clamped_not_zero": (
        "if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0.0;",
        "if (x < 0) x = 0; if (y < 0) y = 0; if (z < 0) z = 0;"
        " if (x >= nx) x = nx - 1; if (y >= ny) y = ny - 1; if (z >= nz) z = nz - 1;"),
    "sample_std": ("*stdv = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;",
                   "*stdv = n > 1 ? sqrt(q / (double)(n - 1)) : 0.0;"),
    "ddof_ignored": ("*stdv = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;", "*stdv = sqrt(q / (double)n);"),
    "threshold_not_strict": ("if (v > T) mask[word] |= bit;", "if (v >= T) mask[word] |= bit;"),
    "bit_order_reversed": ("const uint32_t bit = 1u << (z % 32);\n                if (v > T)",
                           "const uint32_t bit = 1u << (31 - z % 32);\n                if (v > T)"),
    "window_tail_off_by_one": ("for (int64_t z = e * wz; z < nz && z < (e + 1) * wz; ++z)",
                               "for (int64_t z = e * wz; z < nz && z <= (e + 1) * wz; ++z)"),
    "detect_drops_last_filter": ("for (int f = 0; f < nf; ++f) {\n        const double *gxy",
                                 "for (int f = 0; f < nf - (nf > 1); ++f) {\n        const double *gxy"),
}


# slips in the per-voxel local statistics, caught by tests/test_oracle_local_pins.py
LOCAL_MUTANTS = {
    "local_box_clipped_short": ("x1 = x + sx >= nx ? nx - 1 : x + sx;",
                                "x1 = x + sx >= nx ? nx - 2 : x + sx;"),
    "local_y_uses_z_half_width": ("y0 = y - sy < 0 ? 0 : y - sy, y1 = y + sy >= ny ? ny - 1 : y + sy;",
                                  "y0 = y - sz < 0 ? 0 : y - sz, y1 = y + sz >= ny ? ny - 1 : y + sz;"),
    "local_sample_std": ("stdv[i] = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;",
                         "stdv[i] = n > 1 ? sqrt(q / (double)(n - 1)) : 0.0;"),
    "local_ddof_ignored": ("stdv[i] = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;",
                           "stdv[i] = sqrt(q / (double)n);"),
}


# slips in the weighted convolution, caught by tests/test_oracle_weighted_pins.py
WEIGHTED_MUTANTS = {
    "weighted_product_drops_w": ("pw[q] = (double)d[v] * (double)w[v];", "pw[q] = (double)d[v];"),
    "weighted_den_modes_swapped": ("if (den_mode == 0) {\n        passes3(ww,",
                                   "if (den_mode != 0) {\n        passes3(ww,"),
    "weighted_zero_den_gives_one": ("out[v] = den[v] != 0.0 ? num[v] / den[v] : 0.0;",
                                    "out[v] = den[v] != 0.0 ? num[v] / den[v] : 1.0;"),
}


# slips in the selection and OR that the wrapper composes for the sliding and
# the weighted detect (oracle/__init__.py), caught by the pins of each
PY_MUTANTS = {
    "local_detect_sign_flipped": ("thr = mv + k * sv", "thr = mv - k * sv",
                                  "test_oracle_local_pins.py"),
    "local_detect_variance_not_std": ("thr = mv + k * sv", "thr = mv + k * sv * sv",
                                      "test_oracle_local_pins.py"),
    "local_detect_not_strict": ("fire_f = cv > thr", "fire_f = cv >= thr",
                                "test_oracle_local_pins.py"),
    "local_detect_drops_last_filter": ("fire = fire_f.any(axis=0)", "fire = fire_f[:-1].any(axis=0)",
                                       "test_oracle_local_pins.py"),
    "local_detect_drops_first_filter": ("fire = fire_f.any(axis=0)", "fire = fire_f[1:].any(axis=0)",
                                        "test_oracle_local_pins.py"),
    "weighted_detect_sign_flipped": ("thr = mb + k * sb", "thr = mb - k * sb",
                                     "test_oracle_weighted_pins.py"),
    "weighted_detect_not_strict": ("ff = c > thr", "ff = c >= thr", "test_oracle_weighted_pins.py"),
    "weighted_detect_drops_last_filter": ("        fire |= ff\n",
                                          "        fire |= ff if f + 1 < nf else False\n",
                                          "test_oracle_weighted_pins.py"),
    "weighted_detect_window_index_reversed": (
        "wi = [np.arange(n) // wn for n, wn in zip(d.shape, window)]",
        "wi = [np.arange(n)[::-1] // wn for n, wn in zip(d.shape, window)]",
        "test_oracle_weighted_pins.py"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(LOCAL_MUTANTS) + sorted(WEIGHTED_MUTANTS)
                         + sorted(PY_MUTANTS))
def test_pins_catch_planted_slip(tmp_path, name):
    local = name in LOCAL_MUTANTS
    weighted = name in WEIGHTED_MUTANTS
    py = name in PY_MUTANTS
    if py:
        old, new, pins = PY_MUTANTS[name]
    else:
        old, new = (LOCAL_MUTANTS[name] if local else WEIGHTED_MUTANTS[name] if weighted
                    else MUTANTS[name])
        pins = ("test_oracle_local_pins.py" if local else
                "test_oracle_weighted_pins.py" if weighted else "test_oracle_pins.py")
    dst = tmp_path / "oracle_mutant"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = dst / ("__init__.py" if py else "sf_oracle.c")
    text = src.read_text()
    assert old in text and (not py or text.count(old) == 1), f"mutation site for {name} not found"
    src.write_text(text.replace(old, new, 1))
    # the mutant must compile: a build error would count as "caught" otherwise
    if py:
        compile(src.read_text(), str(src), "exec")
    else:
        cc = subprocess.run(["gcc", "-std=c99", "-fopenmp", "-fsyntax-only", str(src)],
                            capture_output=True, text=True)
        assert cc.returncode == 0, cc.stderr
    env = dict(os.environ, SF_ORACLE_DIR=str(dst))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", pins)],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"pins did not catch {name}:\n{res.stdout[-2000:]}"
