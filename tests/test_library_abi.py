"""The C-ABI library builds, loads and exports every symbol include/lrfsi.h
declares (CPU only: no compute call)."""
import os
import subprocess

from paper_2008_10275_gb300 import build, lrfsi


def test_library_builds_and_exports_declared_symbols():
    path = build.build()
    assert os.path.exists(path)
    lib = lrfsi.load()
    syms = lrfsi.declared_symbols()
    assert len(syms) >= 18
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(syms) <= exported


def test_last_error_and_launch_counter_need_no_gpu():
    lib = lrfsi.load()
    assert isinstance(lib.lrfsi_last_error(), bytes)
    assert lrfsi.kernel_launches() >= 0
