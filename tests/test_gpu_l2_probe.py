"""rpp_l2_read_probe, the L2 read-bandwidth probe against which the
apparent-pair pass (whose distance rows stay in L2) is measured. The probe
adds the sum of every 32-bit word it reads to a counter, so the counter must
equal reps times the buffer's word sum (mod 2^32): every load of every
repetition was made, over the whole buffer, including the ragged tail of a
size that is not a multiple of the grid's stride."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _probe(rpp, torch, words, reps, blocks):
    buf = torch.from_numpy(words.view(np.int32)).cuda()
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    rpp.rpp_l2_read_probe(buf, reps, blocks, sink)
    torch.cuda.synchronize()
    got = int(sink.cpu().numpy().view(np.uint32)[0])
    want = int(reps) * int(words.astype(np.uint64).sum()) % (1 << 32)
    return got, want


def test_l2_probe_reads_every_word_reps_times():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as rpp

    rng = np.random.default_rng(7)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # (16-byte elements, reps, blocks): one element; fewer elements than
    # threads; ragged tails of the four-load steps; the 16 MB size of the
    # 2000-point distance matrix over the grid shapes the bench times
    cases = ((1, 1, 1), (1000, 3, 1), (4 * 512 * 2 + 5, 2, 2), (123457, 5, sms),
             ((16 << 20) // 16, 4, 2 * sms), ((16 << 20) // 16, 3, 8 * sms))
    for n16, reps, blocks in cases:
        words = rng.integers(0, 1 << 32, size=4 * n16, dtype=np.uint64).astype(np.uint32)
        got, want = _probe(rpp, torch, words, reps, blocks)
        assert got == want, (n16, reps, blocks)


def test_l2_probe_rejects_host_memory_and_foreign_sizes():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as rpp
    from paper_2003_07989_gb300 import _native as N

    L = N.lib()
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    host = torch.zeros(64, dtype=torch.int32).pin_memory()
    assert L.rpp_l2_read_probe(host.data_ptr(), 256, 1, 1, sink.data_ptr(), None) == N.RPP_E_INVALID
    dev = torch.zeros(64, dtype=torch.int32, device="cuda")
    assert L.rpp_l2_read_probe(dev.data_ptr(), 256, 1, 1, host.data_ptr(), None) == N.RPP_E_INVALID
    with pytest.raises(ValueError):
        rpp.rpp_l2_read_probe(host, 1, 1, sink)
    assert int(sink.item()) == 0
