"""The allocation-free compressor (qsim_compress_block_noalloc).

Some callers cannot let the library call cudaMalloc when they compress a
block: their framework already owns the device memory through its own pool,
or they must keep a fixed footprint once started, or they run in a loop
where an allocation would synchronise the device. The no-alloc entry point
serves them from a fixed device array. Here it must give the same stream,
byte for byte, as qsim_compress_block and as the CPU oracle's encoder, on
two calls in a row (the second call finds the first call's leftovers in the
shared array), also when it is the first call of the library in a fresh
process, and reject blocks larger than its fixed scratch covers; the library's
own allocation count (qsim_alloc_count) must not move across these calls. This
file is collected last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(5, 10, 1e-3), (12, 16, 1e-3), (16, 20, 1e-2), (22, 28, 1e-3)]


def test_noalloc_matches_compress_block_on_consecutive_calls():
    for call in range(2):
        for m, n_equiv, eps in CASES:
            x = torch.from_numpy(inputs.gaussian_block(m, n_equiv, 40 + m + call)).cuda()
            eb = eps * 2.0 ** (-n_equiv / 2)
            ref, nref = qsim.compress_block(x, m, eb)
            out = torch.full((qsim.worst_case_bytes(m),), 0xAB, dtype=torch.uint8, device="cuda")
            allocs = qsim.alloc_count()
            rc, nb = qsim.compress_block_noalloc(x, m, eb, out)
            assert qsim.alloc_count() == allocs  # nothing allocated by the library for this call
            assert rc == qsim.OK, qsim.lib().qsim_last_error()
            assert nb == nref
            assert torch.equal(out[:nb], ref[:nref]), (call, m)
            assert out[:nb].cpu().numpy().tobytes() == oracle.qsz_encode(x.cpu().numpy(), m, eb), (call, m)


def test_noalloc_limits_and_capacity():
    m = qsim.NOALLOC_MAX_M + 1
    x = torch.zeros(1 << m, dtype=torch.complex64, device="cuda")
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    rc, _ = qsim.compress_block_noalloc(x, m, 1e-6, out)
    assert rc == qsim.E_INVALID
    m = 14
    x = torch.from_numpy(inputs.gaussian_block(m, 20, 9)).cuda()
    ref, nref = qsim.compress_block(x, m, 1e-6)
    out = torch.empty(nref - 16, dtype=torch.uint8, device="cuda")
    rc, needed = qsim.compress_block_noalloc(x, m, 1e-6, out)
    assert rc == qsim.E_CAPACITY and needed == nref
    # and the next call is unaffected by the failed one
    out = torch.empty(nref, dtype=torch.uint8, device="cuda")
    rc, nb = qsim.compress_block_noalloc(x, m, 1e-6, out)
    assert rc == qsim.OK and nb == nref and torch.equal(out, ref[:nref])


CHILD = """
import sys
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2410_14088_gb300 import inputs, qsim
torch.cuda.set_device(0)
m, eb = 13, 1e-3 * 2.0 ** -9
allocs = qsim.alloc_count()
for call in range(2):
    x = torch.from_numpy(inputs.gaussian_block(m, 18, 70 + call)).cuda()
    out = torch.zeros(qsim.worst_case_bytes(m), dtype=torch.uint8, device="cuda")
    rc, nb = qsim.compress_block_noalloc(x, m, eb, out)
    assert rc == qsim.OK, qsim.lib().qsim_last_error()
    assert out[:nb].cpu().numpy().tobytes() == oracle.qsz_encode(x.cpu().numpy(), m, eb), call
# the library made no allocation of its own for these calls (torch allocated the tensors)
assert qsim.alloc_count() == allocs, (allocs, qsim.alloc_count())
print("fresh-process no-alloc ok")
"""


def test_noalloc_first_call_in_a_fresh_process():
    # the device address of the fixed array is looked up by the first call on a device: run that call as
    # the first call of the library in a new process, twice in a row, against the oracle's stream
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", CHILD, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process no-alloc ok" in r.stdout
