"""The oracle's pins catch plausible mistakes.  Each mutant below is a copy
of oracle/fasthog_oracle.c with one mistake planted (a flipped sign, an
off-by-one index, a transposed operand, a dropped term, a wrong tie or
boundary rule); it is compiled on the CPU and the oracle pin tests run
against it in a child process (ORACLE_LIB names the mutant's library).  Every
mutant must make at least one pin fail.  No GPU is involved: mistakes are
planted only in the oracle, on the CPU."""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fasthog_oracle.c")
PIN_FILES = ["tests/test_oracle_score.py", "tests/test_oracle_integral.py", "tests/test_oracle_binmap.py",
             "tests/test_oracle_soft.py", "tests/test_oracle_lut.py"]

# (name, text in the oracle, replacement): the first occurrence is replaced
MUTANTS = [
    ("eq1_dy_sign", "int dy = down - up;", "int dy = up - down;"),
    ("eq1_one_sided_dx", "int left = img[y * pitch + (long)channels * (x - 1) + c];",
     "int left = img[y * pitch + (long)channels * (x) + c];"),
    ("channel_tie_to_higher", "if (mag > best_mag) { /* strict: ties keep the lower channel */",
     "if (mag >= best_mag) {"),
    ("upper_half_takes_minus_x", "return dy > 0 || (dy == 0 && dx > 0);", "return dy > 0 || (dy == 0 && dx < 0);"),
    ("sector_boundary_open", "return cross_sign(k, nb, dx, dy) >= 0;", "return cross_sign(k, nb, dx, dy) > 0;"),
    ("table_transposed", "lut[(dy + ORACLE_DMAX) * ORACLE_LUT_SIDE + (dx + ORACLE_DMAX)]",
     "lut[(dx + ORACLE_DMAX) * ORACLE_LUT_SIDE + (dy + ORACLE_DMAX)]"),
    ("integral_drops_first_row", "plane[(long)y * W + x] = row + (y > 0 ? plane[(long)(y - 1) * W + x] : 0);",
     "plane[(long)y * W + x] = row + (y > 1 ? plane[(long)(y - 1) * W + x] : 0);"),
    ("corner_off_by_one", "long v1 = ii_at(ii, W, H, b, x0 - 1, y0 - 1);", "long v1 = ii_at(ii, W, H, b, x0, y0 - 1);"),
    ("corner_sign", "(int32_t)(v4 + v1 - v2 - v3)", "(int32_t)(v4 - v1 - v2 + v3)"),
    ("cell_short_column", "for (int x = i * stride; x < i * stride + cell; ++x) {",
     "for (int x = i * stride; x < i * stride + cell - 1; ++x) {"),
    ("score_drops_bias", "double acc = bias;", "double acc = 0.0;"),
    ("score_feature_transposed", "acc += w[((long)j * cells_x + i) * nb + b] *",
     "acc += w[((long)i * cells_y + j) * nb + b] *"),
    ("detect_strict", "if (v >= thr) {", "if (v > thr) {"),
    ("decimate_odd_column", "src[(long)(2 * y) * pitch + (long)(2 * x) * channels + c]",
     "src[(long)(2 * y) * pitch + (long)(2 * x + 1) * channels + c]"),
    ("block_norm_drops_eps", "double norm = sqrt(ss + eps * eps);", "double norm = sqrt(ss);"),
    ("soft_votes_swapped", "v[k0] += q - a;", "v[k0] += a;"),
    ("soft_centre_shift", "double t = phi * (double)nb / ORACLE_TWO_PI - 0.5;",
     "double t = phi * (double)nb / ORACLE_TWO_PI;"),
    ("channel_by_l1_norm", "long mag = (long)dx * dx + (long)dy * dy;",
     "long mag = (long)(dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);"),
    ("block_cells_transposed", "int ci = i + (q & 1) * r, cj = j + (q >> 1) * r;",
     "int ci = i + (q >> 1) * r, cj = j + (q & 1) * r;"),
    ("detect_drops_stride", "xs[n] = px * stride;", "xs[n] = px;"),
    ("soft_vote_truncated", "int a = (int)floor(x + 0.5);", "int a = (int)floor(x);"),
    ("plus_x_ray_in_lower_half", "static int in_upper_half(int dx, int dy) { return dy > 0 || (dy == 0 && dx > 0); }",
     "static int in_upper_half(int dx, int dy) { return dy > 0; }"),
    ("boundary_cross_sign_flipped", "long cr = c * dy - s * dx;", "long cr = s * dx - c * dy;"),
    ("integral_row_sum_not_reset", "for (int y = 0; y < H; ++y) {\n            int32_t row = 0;",
     "int32_t row = 0;\n        for (int y = 0; y < H; ++y) {"),
    ("corner3_off_by_one", "long v3 = ii_at(ii, W, H, b, x0 - 1, y1);", "long v3 = ii_at(ii, W, H, b, x0, y1);"),
    ("window_cells_unit_step_x", "(double)cells[((long)(py + j * r) * ncx + (px + i * r)) * nb + b];",
     "(double)cells[((long)(py + j * r) * ncx + (px + i)) * nb + b];"),
    ("window_cells_unit_step_y", "(double)cells[((long)(py + j * r) * ncx + (px + i * r)) * nb + b];",
     "(double)cells[((long)(py + j) * ncx + (px + i * r)) * nb + b];"),
]


def build_mutant(workdir, name, old, new):
    src = open(SRC).read()
    assert old in src, f"{name}: the text to mutate is not in the oracle"
    path_c = os.path.join(workdir, f"{name}.c")
    path_so = os.path.join(workdir, f"lib{name}.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new, 1))
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-D_DEFAULT_SOURCE", "-shared",
                    "-fPIC", "-o", path_so, path_c, "-lm"], check=True, capture_output=True)
    return path_so


def run_pins(lib):
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_mutant_is_caught(tmp_path):
    libs = {name: build_mutant(str(tmp_path), name, old, new) for name, old, new in MUTANTS}
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = dict(zip(libs, ex.map(run_pins, libs.values())))
    missed = [name for name, (rc, _) in results.items() if rc == 0]
    assert not missed, f"pins did not catch: {missed}"
    assert all(rc == 1 for rc, _ in results.values()), {n: out for n, (rc, out) in results.items() if rc != 1}


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: an unchanged copy of the oracle passes every pin."""
    lib = build_mutant(str(tmp_path), "unchanged", "int dy = down - up;", "int dy = down - up;")
    rc, out = run_pins(lib)
    assert rc == 0, out
