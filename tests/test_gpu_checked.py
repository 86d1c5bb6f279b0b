"""The checked build runs the small-graph GPU suite clean (needs a GB300).

libn2v_checked.so is the sampler compiled with -DN2V_CHECKED: on the device
it verifies that every special position lies in N(v) and every spill index
in the warp's spill area, that kept specials come in increasing position,
that window searches stay inside their window and bulk copies inside their
buffer, that exactly one of a block step's four ranges holds the draw, that
every chosen index and vertex is in range, and that every stored total of a
stored transition table equals the on-the-fly total.  A failed check sets a
bit of the status word that n2v_stream_status reports as N2V_ERR_INTERNAL;
nothing traps.  The GPU parity tests read the status after every call, so
running them in a child process with N2V_CHECKED=1 checks both the rows and
the self-checks.
"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def run_checked(args: list[str]) -> subprocess.CompletedProcess:
    env = dict(os.environ, N2V_CHECKED="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *args], cwd=REPO,
                          env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=1800)


def test_checked_library_is_the_one_loaded():
    code = ("from paper_1805_00280_gb300 import n2v; import os; "
            "assert n2v.checked(); assert os.path.basename(n2v.lib()._name) == 'libn2v_checked.so'; "
            "print(n2v.n2v_strerror(n2v.N2V_ERR_INTERNAL))")
    r = subprocess.run([sys.executable, "-c", code], cwd=REPO, env=dict(os.environ, N2V_CHECKED="1"),
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "self-check" in r.stdout


def test_small_graph_suite_clean_under_self_checks():
    r = run_checked(["tests/test_gpu_parity.py", "-k",
                     "small_graphs or rmat14 or long_lists or isolated or split_ranges or er_full",
                     "tests/test_gpu_stored.py", "tests/test_gpu_sweeps.py"])
    assert r.returncode == 0, r.stdout[-5000:]
