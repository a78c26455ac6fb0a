"""The oracle's memory accesses under AddressSanitizer (host only).

The oracle keeps small fixed-size tables on the stack (pairs per program, the IBK neighbour
list); an access past one of them would leave its results resting on whatever the stack held.
This test builds a sanitized copy of the same C sources and runs the oracle's own pin tests
against it in a child process -- among them the transfer protocol's pooled fits of 96 and 128
pairs (Sec. 5, Table 2) and IBK predictions over up to 257 training rows.  Any out-of-bounds
read or write aborts the child with a report."""
import os
import subprocess
import sys

import pytest

import oracle

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _libasan():
    try:
        out = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True,
                             check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return out if os.path.isabs(out) and os.path.exists(out) else None


def test_oracle_pins_are_clean_under_address_sanitizer(tmp_path):
    asan = _libasan()
    if asan is None:
        pytest.skip("gcc has no AddressSanitizer runtime here")
    so = oracle.build(sanitize=True)
    env = dict(os.environ, LD_PRELOAD=asan, RS_ORACLE_SO=so,
               ASAN_OPTIONS=f"detect_leaks=0:halt_on_error=1:log_path={tmp_path / 'asan'}")
    tests = [os.path.join(_ROOT, "tests", f) for f in
             ("test_oracle_ibk_pins.py", "test_oracle_transfer_pins.py", "test_oracle_pins.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *tests],
                       cwd=_ROOT, env=env, capture_output=True, text=True, timeout=900)
    reports = "".join(f.read_text()[:4000] for f in tmp_path.glob("asan*"))
    assert not reports, reports
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
