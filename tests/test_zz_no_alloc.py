"""Allocation-free generalized Lanczos (tb_generalized_lanczos_noalloc).

Some callers of this library cannot allocate GPU memory while they call it:
their device memory is already handed to another allocator, or their loop
must not touch the allocator at all.  For them the library offers one entry
point whose scratch is a fixed device array inside the library instead of
cudaMalloc.  These checks call it through the C ABI and compare it with the
allocating tb_generalized_lanczos, to the tolerance of the Lanczos parity
test, on two calls in a row (the shared array keeps the previous call's
contents), with host and device outputs; a request larger than the array
must be refused before any device work.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_1202_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def handle(P):
    from tbinputs import si_system
    return P.tb_create_system(si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0))


def _close(x, y, tol=1e-8):
    return np.abs(np.asarray(x) - np.asarray(y)).max() <= tol * max(1.0, np.abs(np.asarray(y)).max())


def test_noalloc_matches_allocating_entry_point(P, handle):
    ref = {j: P.tb_generalized_lanczos(handle, j, 60) for j in (9, 130)}
    # two calls in a row for the same column, then another column and back,
    # so every call starts from the previous call's leftovers in the array
    for j in (9, 9, 130, 9):
        a, b, nrm = P.tb_generalized_lanczos_noalloc(handle, j, 60)
        a0, b0, n0 = ref[j]
        assert _close(a, a0) and _close(b, b0) and _close(nrm[0], n0)
        assert np.all(b[1:] > 0)


def test_noalloc_device_outputs(P, handle):
    import torch
    a0, b0, n0 = P.tb_generalized_lanczos(handle, 57, 40)
    for _ in range(2):
        out = (torch.zeros(40, dtype=torch.float64, device="cuda"),
               torch.zeros(41, dtype=torch.float64, device="cuda"),
               torch.zeros(1, dtype=torch.float64, device="cuda"))
        a, b, nrm = P.tb_generalized_lanczos_noalloc(handle, 57, 40, out=out)
        assert _close(a.cpu().numpy(), a0) and _close(b.cpu().numpy(), b0) and _close(nrm.item(), n0)


def test_noalloc_rejects_request_beyond_scratch(P, handle):
    with pytest.raises(P.TBError) as e:
        P.tb_generalized_lanczos_noalloc(handle, 9, 3_000_000)
    assert e.value.status == 10
    # the refusal leaves the array usable
    a, b, nrm = P.tb_generalized_lanczos_noalloc(handle, 9, 20)
    a0, b0, n0 = P.tb_generalized_lanczos(handle, 9, 20)
    assert _close(a, a0) and _close(b, b0)


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import paper_1002_1202_gb300 as P
from tbinputs import si_system
torch.cuda.init()
P.load_library()
h = P.tb_create_system(si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0))
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
out = (np.zeros(30), np.zeros(31), np.zeros(1))
P.tb_generalized_lanczos_noalloc(h, 9, 30, out=out)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert np.all(out[1][1:] > 0) and out[2][0] > 0
print("FREE", free0, free1)
"""


def test_noalloc_first_call_in_fresh_process_allocates_nothing(P):
    """In a new process, after tb_create (which allocates), the first call of
    the allocation-free entry point must leave the device's free memory
    unchanged: the fixed array and the call's kernels were placed on the
    device by tb_create, not by this call."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("FREE")][-1].split()
    assert int(line[1]) == int(line[2]), line
