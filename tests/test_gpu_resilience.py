"""Checkpoint / resume and failure detection.

* A checkpoint is a simulation's state plus its level (SP_SURF_STATE +
  SP_SURF_LEVEL); a fresh grid restored from it continues bit-exactly (the
  paper's surfaces are natural checkpoints, Sec. 7).
* Failure detection: a region whose completion is never reported to its
  successors (a failure injected from the host, SP_OPT_FAULT_DROP_RELEASE)
  leaves the device queue waiting; every wait is bounded, so the launch ends
  with SP_ETIMEOUT after the wait limit, the context stays usable, and the
  run is repeated from its checkpoint (the paper's policy: stop, repair,
  continue, Sec. 4).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()


def _params(n, steps):
    return sp.make_params(n, dt=0.25, lam=2.0, eta=1.0, nu=2.0, tau0=10.0, tau_ref=10.0 + steps * 0.25)


def _bits_equal(x, y):
    return all(np.array_equal(np.ascontiguousarray(a).view(np.uint32), np.ascontiguousarray(b).view(np.uint32))
               for a, b in zip(x, y))


def test_checkpoint_resume_is_bit_exact():
    n, first, second = (32, 24, 40), 42, 54
    p = _params(n, first + second)
    st = inputs.initial_state(n, 7, "phase")
    ref = sp.Grid([p])
    try:
        ref.write_state(0, *st)
        ref.plan(base_B=8)
        ref.evolve(first + second)
        want = ref.read_state(0)
    finally:
        ref.close()
    a = sp.Grid([p])
    try:
        a.write_state(0, *st)
        a.plan(base_B=8)
        a.evolve(first)
        ckpt_state, ckpt_level = a.read_state(0), a.level(0)
    finally:
        a.close()
    assert ckpt_level == first
    b = sp.Grid([p])
    try:
        b.write_state(0, *ckpt_state)
        b.set_level(0, ckpt_level)
        b.plan(base_B=8)
        b.evolve(second)
        got = b.read_state(0)
        assert b.level(0) == first + second
    finally:
        b.close()
    assert _bits_equal(got, want)


def test_dropped_release_times_out_and_the_run_recovers():
    n, steps = (32, 32, 32), 16
    p = _params(n, steps)
    st = inputs.initial_state(n, 3, "phase")
    mono = sp.Grid([p])
    try:
        mono.write_state(0, *st)
        mono.evolve(steps, sp.SP_MONOLITHIC)
        want = mono.read_state(0)
    finally:
        mono.close()
    g = sp.Grid([p])
    try:
        g.plan(base_B=8)
        g.set_option(sp.SP_OPT_WAIT_LIMIT_NS, 200_000_000)  # 0.2 s
        g.set_option(sp.SP_OPT_FAULT_DROP_RELEASE, 5)       # a band-0 pyramid
        g.write_state(0, *st)
        g.set_level(0, 0)
        with pytest.raises(sp.SpError) as err:
            g.evolve(steps)
        assert err.value.code == sp.SP_ETIMEOUT
        # repair and continue from the checkpoint: same handle, same context
        g.set_option(sp.SP_OPT_FAULT_DROP_RELEASE, -1)
        g.write_state(0, *st)
        g.set_level(0, 0)
        g.evolve(steps)
        got = g.read_state(0)
    finally:
        g.close()
    assert _bits_equal(got, want)


def test_options_are_validated():
    p = _params((16, 16, 16), 8)
    g = sp.Grid([p])
    try:
        for opt, bad in ((sp.SP_OPT_WAIT_LIMIT_NS, 10), (sp.SP_OPT_FAULT_DROP_RELEASE, -2), (sp.SP_OPT_GRAPHS, 2),
                         (99, 0)):
            with pytest.raises(sp.SpError):
                g.set_option(opt, bad)
        with pytest.raises(sp.SpError):
            g.set_level(0, -1)
    finally:
        g.close()
