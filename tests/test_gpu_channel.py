"""Channel semantics on the GPU (Sec. 3.2.2 Channel API, Sec. 3.1 tag counters).

* payload delivered = payload sent, bit for bit, message by message, in order;
* a receive posted before its send gets the payload straight into its buffer
  (the slot stays untouched), mixed in any order with slot-path and zero-copy
  messages;
* zero-copy receives leave message n in the slot of parity n & 1 and hold the
  slot until the next receive or channel_release: a send that would overwrite
  it waits (bounded) instead;
* a size mismatch is reported as JACOBI_ESEQ;
* a waiting receive with no matching send times out (bounded wait) with
  JACOBI_ETIMEDOUT instead of hanging, and the context stays usable; a posted
  receive still waiting for its send is reported as JACOBI_EAGAIN;
* the on-device ping-pong completes for 8 B .. 4 MB and leaves the payload.
"""
import pytest

import paper_2102_12416_gb300 as jg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class _DevBuf:
    """Raw device bytes viewed as a torch tensor (no copy, no allocation)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _view(ptr, n):
    return torch.as_tensor(_DevBuf(ptr, n), device="cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2102_12416_gb300 import _build
    _build.build()
    jg.load()


@pytest.fixture
def solver(monkeypatch):
    monkeypatch.setenv("JACOBI_WAIT_MS", "200")
    s = jg.Jacobi3D((32, 32, 32), ("count", (2, 2, 2)), "f64")
    yield s
    s.close()


def _payload(n_bytes, tag):
    g = torch.Generator().manual_seed(1000 + tag)
    return torch.randint(0, 256, (n_bytes,), dtype=torch.uint8, generator=g).cuda()


def test_ordered_exactly_once(solver):
    ch = jg.channel_open(solver.h, 7, 0, 1, 1 << 16)
    try:
        dst = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
        for k, n in enumerate([16, 4096, 65536, 48, 1024, 8, 12345]):
            src = _payload(n, k)
            jg.channel_send(ch, 0, src.data_ptr(), n)
            jg.channel_recv(ch, 1, dst.data_ptr(), n)
            jg.channel_sync(ch)
            assert torch.equal(dst[:n], src), k
        # both directions interleaved
        for k in range(6):
            a, b = _payload(256, 50 + k), _payload(256, 80 + k)
            jg.channel_send(ch, 0, a.data_ptr(), 256)
            jg.channel_send(ch, 1, b.data_ptr(), 256)
            jg.channel_recv(ch, 1, dst.data_ptr(), 256)
            got_b = dst[:256].clone()
            jg.channel_recv(ch, 0, dst.data_ptr(), 256)
            jg.channel_sync(ch)
            assert torch.equal(got_b, a) and torch.equal(dst[:256], b)
    finally:
        jg.channel_close(ch)


def test_two_in_flight_then_receive(solver):
    ch = jg.channel_open(solver.h, 8, 2, 3, 4096)
    try:
        m0, m1 = _payload(4096, 1), _payload(4096, 2)
        jg.channel_send(ch, 2, m0.data_ptr(), 4096)
        jg.channel_send(ch, 2, m1.data_ptr(), 4096)
        d0 = torch.zeros(4096, dtype=torch.uint8, device="cuda")
        d1 = torch.zeros_like(d0)
        jg.channel_recv(ch, 3, d0.data_ptr(), 4096)
        jg.channel_recv(ch, 3, d1.data_ptr(), 4096)
        jg.channel_sync(ch)
        assert torch.equal(d0, m0) and torch.equal(d1, m1)
    finally:
        jg.channel_close(ch)


def test_zero_copy_slot(solver):
    ch = jg.channel_open(solver.h, 9, 0, 4, 1024)
    try:
        for n in range(4):
            m = _payload(1024, 10 + n)
            jg.channel_send(ch, 0, m.data_ptr(), 1024)
            jg.channel_recv(ch, 4, None, 1024)
            jg.channel_sync(ch)
            slot = _view(jg.channel_slot(ch, 4, n & 1), 1024)
            assert torch.equal(slot, m), n
    finally:
        jg.channel_close(ch)


def test_size_mismatch_is_seq_error(solver):
    ch = jg.channel_open(solver.h, 10, 5, 6, 1024)
    try:
        m = _payload(512, 3)
        d = torch.zeros(1024, dtype=torch.uint8, device="cuda")
        jg.channel_send(ch, 5, m.data_ptr(), 512)
        jg.channel_recv(ch, 6, d.data_ptr(), 1024)
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_sync(ch)
        assert e.value.code == jg.JACOBI_ESEQ
    finally:
        jg.channel_close(ch)


def test_recv_without_send_times_out(solver):
    ch = jg.channel_open(solver.h, 11, 0, 7, 256)
    try:
        jg.channel_recv(ch, 7, None, 256)  # zero-copy: waits on the device; nothing was sent
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_sync(ch)
        assert e.value.code == jg.JACOBI_ETIMEDOUT
    finally:
        jg.channel_close(ch)
    # the GPU context is still usable afterwards
    solver.step(2)
    solver.sync()


def test_posted_receive_gets_payload_directly(solver):
    n = 4096
    ch = jg.channel_open(solver.h, 13, 0, 1, n)
    try:
        dst = torch.zeros(n, dtype=torch.uint8, device="cuda")
        jg.channel_recv(ch, 1, dst.data_ptr(), n)  # posted before the send
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_sync(ch)
        assert e.value.code == jg.JACOBI_EAGAIN
        m = _payload(n, 40)
        jg.channel_send(ch, 0, m.data_ptr(), n)
        jg.channel_sync(ch)
        assert torch.equal(dst, m)
        # the message went straight to dst: the slot of its parity is untouched
        assert int(_view(jg.channel_slot(ch, 1, 0), n).sum()) == 0
        # posted, slot path, zero-copy and posted again, both directions
        outs = []
        for k in range(8):
            m = _payload(n, 41 + k)
            d = torch.zeros(n, dtype=torch.uint8, device="cuda")
            a, b = (0, 1) if k % 2 == 0 else (1, 0)
            mode = k % 3
            if mode == 0:
                jg.channel_recv(ch, b, d.data_ptr(), n)
                jg.channel_send(ch, a, m.data_ptr(), n)
            elif mode == 1:
                jg.channel_send(ch, a, m.data_ptr(), n)
                jg.channel_recv(ch, b, d.data_ptr(), n)
            else:
                jg.channel_send(ch, a, m.data_ptr(), n)
                jg.channel_recv(ch, b, None, n)
                parity = sum(1 for j in range(k) if (j % 2 == 0) == (k % 2 == 0)) + (1 if b == 1 else 0)
                jg.channel_sync(ch)
                d.copy_(_view(jg.channel_slot(ch, b, parity & 1), n))
                jg.channel_release(ch, b)
            jg.channel_sync(ch)
            outs.append((d, m))
        for k, (d, m) in enumerate(outs):
            assert torch.equal(d, m), k
        # a posted receive of another size: the send is refused at once
        d = torch.zeros(n, dtype=torch.uint8, device="cuda")
        jg.channel_recv(ch, 1, d.data_ptr(), 1024)
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_send(ch, 0, _payload(512, 3).data_ptr(), 512)
        assert e.value.code == jg.JACOBI_ESEQ
    finally:
        jg.channel_close(ch)


def test_zero_copy_holds_slot_until_released(solver):
    n = 1024
    msgs = [_payload(n, 60 + k) for k in range(3)]
    ch = jg.channel_open(solver.h, 14, 2, 3, n)
    try:
        jg.channel_send(ch, 2, msgs[0].data_ptr(), n)
        jg.channel_recv(ch, 3, None, n)  # message 0 stays in slot 0, held
        jg.channel_send(ch, 2, msgs[1].data_ptr(), n)  # slot 1: free
        jg.channel_send(ch, 2, msgs[2].data_ptr(), n)  # slot 0: held, so this send must wait
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_sync(ch)
        assert e.value.code == jg.JACOBI_ETIMEDOUT
        assert torch.equal(_view(jg.channel_slot(ch, 3, 0), n), msgs[0])
    finally:
        jg.channel_close(ch)
    # released after reading, the same sequence goes through
    ch = jg.channel_open(solver.h, 15, 2, 3, n)
    try:
        jg.channel_send(ch, 2, msgs[0].data_ptr(), n)
        jg.channel_recv(ch, 3, None, n)
        got0 = _view(jg.channel_slot(ch, 3, 0), n).clone()
        jg.channel_release(ch, 3)
        jg.channel_send(ch, 2, msgs[1].data_ptr(), n)
        jg.channel_send(ch, 2, msgs[2].data_ptr(), n)
        d1 = torch.zeros(n, dtype=torch.uint8, device="cuda")
        d2 = torch.zeros_like(d1)
        jg.channel_recv(ch, 3, d1.data_ptr(), n)
        jg.channel_recv(ch, 3, d2.data_ptr(), n)
        jg.channel_sync(ch)
        assert torch.equal(got0, msgs[0]) and torch.equal(d1, msgs[1]) and torch.equal(d2, msgs[2])
    finally:
        jg.channel_close(ch)
    solver.step(2)
    solver.sync()


def test_duplicate_channel_id_rejected(solver):
    ch = jg.channel_open(solver.h, 12, 0, 1, 64)
    try:
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_open(solver.h, 12, 2, 3, 64)
        assert e.value.code == jg.JACOBI_EINVAL
    finally:
        jg.channel_close(ch)


@pytest.mark.parametrize("nbytes,ctas", [(8, 1), (4096, 1), (65536, 2), (1 << 20, 16), (4 << 20, 32)])
def test_pingpong_runs_and_delivers(solver, nbytes, ctas):
    ch = jg.channel_open(solver.h, 20, 0, 1, 4 << 20)
    try:
        # the ping-pong sends each endpoint's parity-1 slot into the peer's parity-0 slot
        a, b = _payload(nbytes, 1), _payload(nbytes, 2)
        _view(jg.channel_slot(ch, 0, 1), nbytes).copy_(a)
        _view(jg.channel_slot(ch, 1, 1), nbytes).copy_(b)
        torch.cuda.synchronize()
        jg.channel_pingpong(ch, nbytes, 10, ctas)
        jg.channel_sync(ch)
        assert torch.equal(_view(jg.channel_slot(ch, 1, 0), nbytes), a)
        assert torch.equal(_view(jg.channel_slot(ch, 0, 0), nbytes), b)
    finally:
        jg.channel_close(ch)


def test_host_staged_and_messaging_forms(solver):
    ch = jg.channel_open(solver.h, 30, 0, 1, 1 << 20)
    try:
        for k, n in enumerate([16, 4096, 1 << 20]):
            src = _payload(n, 200 + k)
            dst = torch.zeros(n, dtype=torch.uint8, device="cuda")
            jg.channel_send_host(ch, 0, src.data_ptr(), n)
            jg.channel_recv_host(ch, 1, dst.data_ptr(), n)
            assert torch.equal(dst, src)
            dst.zero_()
            jg.channel_send_msg(ch, 1, src.data_ptr(), n)
            jg.channel_recv_msg(ch, 0, dst.data_ptr(), n)
            assert torch.equal(dst, src)
        # the receive can only be posted once the metadata message is there
        d = torch.zeros(256, dtype=torch.uint8, device="cuda")
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_recv_msg(ch, 1, d.data_ptr(), 64)
        assert e.value.code == jg.JACOBI_EAGAIN
        m = _payload(64, 7)
        jg.channel_send_msg(ch, 0, m.data_ptr(), 64)
        with pytest.raises(jg.JacobiError) as e:
            jg.channel_recv_msg(ch, 1, d.data_ptr(), 32)
        assert e.value.code == jg.JACOBI_ESEQ
        # the comparison forms leave the device channel's sequence numbers alone
        for k in range(5):
            src = _payload(256, 300 + k)
            jg.channel_send(ch, k % 2, src.data_ptr(), 256)
            jg.channel_recv(ch, 1 - k % 2, d.data_ptr(), 256)
            jg.channel_sync(ch)
            assert torch.equal(d, src)
    finally:
        jg.channel_close(ch)


@pytest.mark.parametrize("bidir", [False, True])
def test_bandwidth_window_runs_and_delivers(solver, bidir):
    n = 1 << 20
    ch = jg.channel_open(solver.h, 31, 2, 3, n)
    try:
        a, b = _payload(n, 11), _payload(n, 12)
        _view(jg.channel_slot(ch, 2, 1), n).copy_(a)
        _view(jg.channel_slot(ch, 3, 1), n).copy_(b)
        torch.cuda.synchronize()
        jg.channel_bandwidth(ch, n, 8, 5, 8, bidir)
        jg.channel_sync(ch)
        assert torch.equal(_view(jg.channel_slot(ch, 3, 0), n), a)
        if bidir:
            assert torch.equal(_view(jg.channel_slot(ch, 2, 0), n), b)
    finally:
        jg.channel_close(ch)
