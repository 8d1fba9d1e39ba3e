"""The serving slab's first-fit allocator against a plain interval model (CPU)."""
import pytest

import synth


@pytest.fixture(scope="module")
def rr():
    from paper_1011_3583_gb300 import build
    build.build()
    import paper_1011_3583_gb300 as rr
    return rr


BASE = 1 << 40


def model_first_fit(free, need):
    """free: sorted list of (start, size); lowest start that fits."""
    for s, z in free:
        if z >= need:
            return s
    return None


def model_free_list(cap, live):
    """Free intervals of [BASE, BASE+cap) given live blocks {start: size}."""
    out, cur = [], BASE
    for s in sorted(live):
        if s > cur:
            out.append((cur, s - cur))
        cur = s + live[s]
    if cur < BASE + cap:
        out.append((cur, BASE + cap - cur))
    return out


def test_arena_matches_first_fit_model(rr):
    cap = 1 << 20
    a = rr.Arena(BASE, cap)
    g = synth.rng(3)
    live = {}
    for step in range(3000):
        if live and g.random() < 0.45:
            addr = list(live)[int(g.integers(0, len(live)))]
            a.free(addr)
            del live[addr]
        else:
            want = int(g.integers(1, 40000))
            need = (want + 255) // 256 * 256
            expect = model_first_fit(model_free_list(cap, live), need)
            if expect is None:
                with pytest.raises(rr.RearrError) as ex:
                    a.alloc(want)
                assert ex.value.status == 2  # REARR_ENOMEM
            else:
                addr = a.alloc(want)
                assert addr == expect and addr % 256 == 0
                live[addr] = need
        st = a.stats()
        assert st["used"] == sum(live.values()) and st["blocks"] == len(live)
        fl = model_free_list(cap, live)
        assert st["largest_free"] == max([z for _, z in fl], default=0)
    for addr in list(live):
        a.free(addr)
    assert a.stats() == dict(used=0, free=cap, largest_free=cap, blocks=0)  # fully coalesced
    a.close()


def test_arena_rejects_unknown_and_double_free(rr):
    a = rr.Arena(BASE, 1 << 16)
    x = a.alloc(100)
    with pytest.raises(rr.RearrError):
        a.free(x + 256)
    a.free(x)
    with pytest.raises(rr.RearrError):
        a.free(x)
    with pytest.raises(rr.RearrError):
        a.alloc(1 << 17)
    a.close()
