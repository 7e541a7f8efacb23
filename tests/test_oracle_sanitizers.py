"""The oracle under AddressSanitizer and UBSan on the host: every mode,
valid and corrupted archives (tests/oracle_asan_driver.c).  Any read or write
outside a buffer, or undefined behaviour, fails the run."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_is_clean_under_asan_and_ubsan():
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "oracle_asan")
        cmd = ["gcc", "-O1", "-g", "-std=gnu11", "-ffp-contract=off", "-fno-omit-frame-pointer",
               "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
               os.path.join(ROOT, "oracle", "gbsz_oracle.c"), os.path.join(ROOT, "tests", "oracle_asan_driver.c"),
               "-o", exe, "-lm"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0 and b"asan" in r.stdout.lower():
            pytest.skip("the sanitizer runtime is not installed: " + r.stdout.decode()[-300:])
        assert r.returncode == 0, r.stdout.decode()[-3000:]
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
        r = subprocess.run([exe], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, env=env, timeout=600)
        out = r.stdout.decode()
        assert r.returncode == 0, out[-4000:]
        assert out.strip().startswith("ok "), out[-2000:]
