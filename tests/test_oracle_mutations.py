"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
never on a GPU), builds it into a temporary library and runs the pin suite
against it in a subprocess; the suite has to fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vspec_oracle.c")

MUTATIONS = {
    "fft_twiddle_sign": ("double ang = -2.0 * VSO_PI", "double ang = 2.0 * VSO_PI"),
    "fir_tap_order": ("ar += h[(long)t * nchan + n] * xr;\n            ai += h[(long)t * nchan + n] * xi;",
                      "ar += h[(long)(P - 1 - t) * nchan + n] * xr;\n            ai += h[(long)(P - 1 - t) * nchan + n] * xi;"),
    "cross_term_sign": ("xi * yr - xr * yi", "xr * yi - xi * yr"),
    "pol_layout": ("long idx = (m * npol + p) * 2;", "long idx = (m * npol + (npol - 1 - p)) * 2;"),
    "hann_sign": ("0.5 - 0.5 * cos(phase)", "0.5 + 0.5 * cos(phase)"),
    "sinc_width": ("/ (double)nchan;\n            h[i] = w * sinc(u);", "/ (double)(2 * nchan);\n            h[i] = w * sinc(u);"),
    "detect_drops_imag": ("acc[k] += xr * xr + xi * xi;", "acc[k] += xr * xr;"),
    "no_accumulation": ("acc[k] += xr * xr + xi * xi;", "acc[k] = xr * xr + xi * xi;"),
    "butterfly_difference": ("out[2 * (k + h)] = er - tr;", "out[2 * (k + h)] = er + tr;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "vspec_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libvspec_oracle_mut.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, VSPEC_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
