"""GPU: rq_copy moves bytes between pinned host and device memory (and within
device memory) with the SMs, exactly: host -> device -> device -> host returns
the original bytes for aligned and unaligned offsets and odd lengths; pageable
host memory, NULL pointers and overlapping ranges are refused."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbytes,off", [(1 << 20, 0), (12345, 3), (17, 1), (4096 * 8 + 8, 8)])
def test_round_trip_is_exact(nbytes, off):
    import torch
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    g = torch.Generator(device="cpu")
    g.manual_seed(nbytes)
    h0 = torch.randint(0, 256, (nbytes + 64,), dtype=torch.uint8, generator=g).pin_memory()
    d1 = torch.zeros(nbytes + 64, dtype=torch.uint8, device="cuda")
    d2 = torch.zeros(nbytes + 64, dtype=torch.uint8, device="cuda")
    h3 = torch.zeros(nbytes + 64, dtype=torch.uint8).pin_memory()
    assert _lib.rq_copy(d1.data_ptr() + off, h0.data_ptr() + off, nbytes) == 0
    assert _lib.rq_copy(d2.data_ptr() + off, d1.data_ptr() + off, nbytes) == 0
    assert _lib.rq_copy(h3.data_ptr() + off, d2.data_ptr() + off, nbytes) == 0
    torch.cuda.synchronize()
    assert torch.equal(h3[off:off + nbytes], h0[off:off + nbytes])
    assert int(h3[:off].sum()) == 0 and int(h3[off + nbytes:].sum()) == 0
    assert torch.equal(d1[off:off + nbytes].cpu(), h0[off:off + nbytes])


def test_refusals():
    import torch
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    pageable = torch.zeros(1024, dtype=torch.uint8)
    d = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    assert _lib.rq_copy(d.data_ptr(), pageable.data_ptr(), 1024) == -2
    assert _lib.rq_copy(pageable.data_ptr(), d.data_ptr(), 1024) == -1
    assert _lib.rq_copy(None, d.data_ptr(), 16) == -1
    assert _lib.rq_copy(d.data_ptr(), None, 16) == -2
    assert _lib.rq_copy(d.data_ptr() + 8, d.data_ptr(), 64) == -1      # overlap
    assert _lib.rq_copy(d.data_ptr(), d.data_ptr(), 0) == 0
    torch.cuda.synchronize()
