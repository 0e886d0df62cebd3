"""Host build of the bit helpers used by the key kernels: the in-register
32 x 32 bit transpose must put bit c of row m at bit m of column c, and the
partition hash must be a bijection (equal keys share a partition, distinct
keys never merge).  The class-split filter's construction is checked the
same way: its key classes are linear, so the round that holds class q
tests exactly the keys whose partner is of class q, and class planes
formed from the row words come out of the transpose as each key's class."""
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


def test_class_split_construction_on_host(tmp_path):
    exe = tmp_path / "class_split_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-x", "c++", os.path.join(HERE, "host", "class_split_test.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
