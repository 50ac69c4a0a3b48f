"""Host logic of the serving load generator, without a GPU: the page-locked output ring
hands a slice to a new job only after every job holding an overlapping slice has been
waited on, and every slice lies inside the ring.  The server is a fake that records the
submitted jobs; the ring is small (96 MB, one and a half largest jobs) so that it wraps
many times, at ragged points."""
import numpy as np

from paper_2304_12745_gb300 import capi, serving


class _FakeServer:
    handle = 1

    def reset_stats(self):
        pass

    def stats(self):
        return {}


def test_ring_slices_are_reused_only_after_their_jobs_were_waited_on(monkeypatch):
    ring_bytes = 96 << 20  # the largest job (1,024 x 32 x 256 complex64) is 64 MB
    buffers, live, seen = [], {}, []

    def fake_pinned(n, dtype):
        a = np.zeros(n, dtype)
        buffers.append(a)
        return a

    def submit(handle, job):
        lo = job.W_out
        hi = lo + job.n_sc * job.K * job.M * 8
        for a, b in live.values():
            assert not (a < hi and lo < b), "an output slice still held by a live job was reused"
        ticket = len(seen)
        live[ticket] = (lo, hi)
        seen.append((lo, hi))
        return ticket

    def wait(handle, ticket, timeout_us):
        live.pop(ticket, None)
        return 0

    monkeypatch.setattr(capi, "precode_serve_submit", submit)
    monkeypatch.setattr(capi, "precode_serve_wait", wait)
    monkeypatch.setattr(serving, "pinned", fake_pinned)
    monkeypatch.setattr(serving, "touch_by_device", lambda *a, **k: None)
    st = serving.poisson_load(_FakeServer(), 40000.0, 0.02, seed=3, ring_bytes=ring_bytes)
    ring = next(b for b in buffers if b.nbytes == ring_bytes)
    base = ring.ctypes.data
    assert st["jobs"] == len(seen) > 100
    assert all(base <= lo < hi <= base + ring_bytes for lo, hi in seen)
    assert sum(hi - lo for lo, hi in seen) > 4 * ring_bytes  # the ring wrapped several times
    assert not live  # every job was waited on at the end
