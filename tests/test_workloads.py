"""The seeded input generators (workloads.py) reproduce the workloads the
measurements and parity tests are stated on: the 256^2 S12 channel (2848
channel cells, the centreline rules), the 1024^2 S16 time-dependent channel
(the 256^2 mask scaled x4), and the 64-problem batch (115,742,904 updates per
batch sweep, sides in [32, 256], S8-S16), each identical from call to call."""
import numpy as np

import workloads as W


def test_channel_workload():
    p = W.config_channel()
    assert (p.nx, p.ny, p.K) == (256, 256, 84)
    st = p.sigma_a + p.sigma_s
    chan = st < 1.0
    assert int(chan.sum()) == 2848
    assert np.allclose(st[chan], 0.2) and np.allclose(st[~chan], 2000.0)
    assert np.allclose(p.sigma_s / st, 0.999)
    assert not p.q.any()
    m = W.channel_mask(256, 2, 8)
    assert np.array_equal(m.reshape(-1), chan)
    # the channel starts at the left wall and reaches the right one
    assert m[:, 0].any() and m[:, -1].any()
    assert np.array_equal(W.config_channel().sigma_a, p.sigma_a)


def test_timedep_workload_is_the_channel_scaled_by_four():
    p = W.config_timedep()
    assert (p.nx, p.ny, p.K) == (1024, 1024, 144)
    chan = (p.sigma_a + p.sigma_s).reshape(1024, 1024) < 1.0
    base = W.channel_mask(256, 2, 8)
    assert np.array_equal(chan, np.kron(base, np.ones((4, 4), dtype=bool)))
    assert int(chan.sum()) == 16 * 2848


def test_batch_workload():
    ps = W.config_batch()
    assert len(ps) == 64
    assert sum(p.N * p.K for p in ps) == 115_742_904
    assert all(32 <= p.nx <= 256 and p.nx == p.ny for p in ps)
    assert {p.K for p in ps} <= {40, 60, 84, 112, 144}
    st = np.concatenate([p.sigma_a + p.sigma_s for p in ps])
    assert st.min() >= 1e-2 * (1 - 1e-12) and st.max() <= 1e4 * (1 + 1e-12)
    again = W.config_batch()
    assert all(np.array_equal(a.sigma_a, b.sigma_a) for a, b in zip(ps, again))
