"""sp_sweep_noalloc: whole-grid steps that allocate no memory.

Callers that may not allocate device memory -- programs that own all device
memory through their own fixed pools, plug-ins that must not grow the
process's footprint, latency-critical paths -- advance a field with this
entry point.  Its only scratch is a pair of fixed device arrays inside the
library.  Here it is checked, through the C ABI, against the allocating entry
point (sp_evolve with SP_MONOLITHIC) on two calls in a row; the two must agree
bit for bit, the bar every GPU-path comparison in this suite uses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

pytestmark = pytest.mark.gpu


def _params(n, steps):
    return sp.make_params(n, dx=1.0, dt=0.25, lam=2.0, eta=1.0, nu=2.0, tau0=10.0, tau_ref=10.0 + steps * 0.25)


def _bits_equal(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint32), np.ascontiguousarray(b).view(np.uint32))


def test_noalloc_sweep_matches_the_allocating_path_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = (32, 24, 40)
    shape = (n[2], n[1], n[0])
    sites = n[0] * n[1] * n[2]
    first, second = 11, 6
    p = _params(n, first + second)
    st = inputs.initial_state(n, 3, "phase")

    # reference: the allocating entry point, same state, same levels
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        g.evolve(first, sp.SP_MONOLITHIC)
        ref1 = g.read_state(0)
        g.evolve(second, sp.SP_MONOLITHIC)
        ref2 = g.read_state(0)
    finally:
        g.close()

    # the caller owns the state; the entry point allocates nothing
    stream = torch.cuda.current_stream()
    buf = torch.from_numpy(sp.pack_state(*st)).cuda()
    phi, pic = buf[:sites], buf[sites:]
    rc = sp.sp_sweep_noalloc(p, phi.data_ptr(), pic.data_ptr(), 0, first, stream.cuda_stream)
    assert rc == sp.SP_OK, sp.sp_strerror(rc)
    stream.synchronize()
    got1 = sp.unpack_state(buf.cpu().numpy(), shape)
    rc = sp.sp_sweep_noalloc(p, phi.data_ptr(), pic.data_ptr(), first, second, stream.cuda_stream)
    assert rc == sp.SP_OK, sp.sp_strerror(rc)
    stream.synchronize()
    got2 = sp.unpack_state(buf.cpu().numpy(), shape)

    assert np.all(np.isfinite(got2[0]))
    for got, ref in ((got1, ref1), (got2, ref2)):
        for a, b, name in zip(got, ref, ("phi", "pi", "c")):
            assert _bits_equal(a, b), f"{name} differs from sp_evolve(SP_MONOLITHIC)"


def test_noalloc_sweep_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = _params((96, 96, 96), 4)  # 884736 sites > 262144
    buf = torch.zeros(3 * 96 ** 3, dtype=torch.complex64, device="cuda")
    rc = sp.sp_sweep_noalloc(p, buf.data_ptr(), buf[96 ** 3:].data_ptr(), 0, 4, 0)
    assert rc == sp.SP_ESCRATCH
    assert "SP_NOALLOC_MAX_SITES" in sp.sp_strerror(rc)
    p = _params((16, 16, 16), sp.SP_NOALLOC_MAX_STEPS + 1)
    rc = sp.sp_sweep_noalloc(p, buf.data_ptr(), buf[16 ** 3:].data_ptr(), 0, sp.SP_NOALLOC_MAX_STEPS + 1, 0)
    assert rc == sp.SP_ESCRATCH
