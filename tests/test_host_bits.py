"""Host build of the bit helpers used by the key kernels: the in-register
32 x 32 bit transpose must put bit c of row m at bit m of column c, and the
partition hash must be a bijection (equal keys share a partition, distinct
keys never merge)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bits_helpers_on_host(tmp_path):
    exe = tmp_path / "bits_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-x", "c++", os.path.join(HERE, "host", "bits_test.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
