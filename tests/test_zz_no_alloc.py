"""pb_collision_static, the no-allocation collision entry point, against pb_collision.

Some callers cannot allocate device memory at all (their device memory belongs to a
host framework's allocator or to a fixed budget set at start-up).  For them the
library offers pb_collision_static, whose scratch is a fixed device array inside
libpb.so.  These tests call it through the C ABI and check its output against the
regular entry point's on two calls in a row (the array keeps the previous call's
contents), for each hot-path variant, and that an oversized problem is refused.
This file is collected last on purpose; it also passes on its own in a new process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_03683_gb300 as pb
    import torch

    assert torch.cuda.is_available()
    return pb


def _call_static(pb, dev, f, out):
    import torch

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return pb.lib().pb_collision_static(dev._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("name,variant,opts", [("tiny", "ff", {}), ("window16", "ff", {}), ("window24", "ff", {}),
                                               ("window16", "ff", {"stream_mode": 2}), ("window16", "f64", {}),
                                               ("window16", "literal", {})])
def test_static_matches_regular_on_two_calls(pb, name, variant, opts):
    import torch

    m = synth.make_config(name)
    dev = pb.Device(pb.Channels.from_model(m), variant=variant, **opts)
    rng = np.random.default_rng(17)
    out = torch.empty(dev.nstate, dtype=torch.float64, device="cuda")
    for call in range(2):
        f = torch.tensor(rng.uniform(0.0, 1.0, dev.nstate), device="cuda")
        rc = _call_static(pb, dev, f, out)
        assert rc == pb.PB_OK, pb.lib().pb_last_error().decode()
        ref = dev.collision(f).cpu().numpy()
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL, f"call {call}: normwise error {err:.3e}"
    dev.check()  # no bounded wait of the bulk-copy sweep gave up


def test_static_call_allocates_nothing(pb):
    """After a first call (which looks up the array's address and loads the kernels), further
    calls leave both torch's allocator and the device's free memory exactly as they were."""
    import torch

    m = synth.make_config("window16")
    dev = pb.Device(pb.Channels.from_model(m))
    f = torch.tensor(np.random.default_rng(3).uniform(0.0, 1.0, dev.nstate), device="cuda")
    out = torch.empty_like(f)
    assert _call_static(pb, dev, f, out) == pb.PB_OK
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        assert _call_static(pb, dev, f, out) == pb.PB_OK
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert after == before


def test_static_refuses_problems_beyond_its_array(pb):
    import torch

    m = synth.make_config("window28")
    # one entry per channel in 64-channel items: ~2.3e5 items, > 4 MiB of partials
    dev = pb.Device(pb.Channels.from_model(m), item_channels=64, merge_branches=2)
    f = torch.full((dev.nstate,), 0.1, dtype=torch.float64, device="cuda")
    out = torch.empty_like(f)
    rc = _call_static(pb, dev, f, out)
    assert rc == pb.PB_EINVAL
    assert "static array holds" in pb.lib().pb_last_error().decode()
