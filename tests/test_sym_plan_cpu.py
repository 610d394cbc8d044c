"""The symmetric kernel's plan (cts_plan_sym), on the CPU: every ordered pair
of carriers of an event is covered exactly once (Eq. 4's sum over j != i,
each unordered pair evaluated once and added to both carriers), the partial
lists hold every written partial exactly once, and a numpy emulation of the
kernel's sign and partial conventions reproduces the FP64 oracle's field."""
import numpy as np
import pytest

import oracle
import paper_2506_09712_gb300 as cts

T, TPB = 64, 4          # carriers per tile, tiles per I block


@pytest.fixture(scope="module")
def lib():
    from paper_2506_09712_gb300 import build
    build.build()
    return cts.load()


def _tiles_of(n):
    return (max(n, 0) + T - 1) // T


def _combos(u, nti):
    """(I tile, J tile, mode) of one unit: mode 2 = both ways, 1 = the tile
    with itself (i sums only), as the kernel evaluates them."""
    slot, si, sj, ib0, ib1, jt0, jt1 = (int(v) for v in u[:7])
    same = si == sj
    for b in range(ib0, ib1):
        bt0 = b * TPB
        vt = min(TPB, nti - bt0)
        for g in range(max(jt0, bt0) if same else jt0, jt1):
            for t in range(vt):
                if same and g < bt0 + TPB:
                    qd = g - bt0
                    if t < qd:
                        yield bt0 + t, g, 2
                    elif t == qd:
                        yield bt0 + t, g, 1
                else:
                    yield bt0 + t, g, 2


CASES = [([300], [0]), ([1], [0]), ([64], [0]), ([65], [0]), ([257], [3]), ([130], [70]),
         ([64], [64]), ([5525], [0]), ([1000, 0, 77, 2000], [0, 5, 77, 300]),
         ([11000], [0]), ([20000], [20000]), ([45000], [0])]


def _pairs(units):
    return units[units[:, 10] == 0]


@pytest.mark.parametrize("n_h,n_e", CASES)
def test_symmetric_plan_covers_every_tile_pair_once(lib, n_h, n_e):
    rc, all_units, tiles, lists, npart = cts.cts_plan_sym(n_h, n_e)
    assert rc == 0
    units = _pairs(all_units)
    for s, (nh, ne) in enumerate(zip(n_h, n_e)):
        th, te = _tiles_of(nh), _tiles_of(ne)
        us = units[units[:, 0] == s]
        if nh <= 0:
            assert len(us) == 0
            continue
        nt = th + te
        M = np.zeros((nt, nt), dtype=np.int64)   # M[a, b]: sources b counted in a's field
        for u in us:
            si, sj = int(u[1]), int(u[2])
            assert not (si == 1 and sj == 0)      # electron rows take no hole tiles
            nti = te if si else th
            oi, oj = (th if si else 0), (th if sj else 0)
            assert 0 <= u[5] < u[6] <= (te if sj else th)
            for ti, tj, mode in _combos(u, nti):
                if mode == 2:
                    M[oi + ti, oj + tj] += 1
                    M[oj + tj, oi + ti] += 1
                else:
                    assert ti == tj and si == sj
                    M[oi + ti, oi + ti] += 1
        assert (M == 1).all(), np.argwhere(M != 1)[:5]
        assert int(us[:, 9].sum()) == 1 and us[0, 9] == 1   # one bookkeeping unit, listed first
    # lists: every partial a unit writes, in exactly one tile's list, in unit order
    written = []
    for u in units:
        s, si, sj, ib0, ib1, jt0, jt1, pi, pj = (int(v) for v in u[:9])
        nti = _tiles_of(n_e[s] if si else n_h[s])
        written += [pi + (b - ib0) * TPB + q for b in range(ib0, ib1) for q in range(TPB)
                    if b * TPB + q < nti]
        written += [pj + g - jt0 for g in range(jt0, jt1)]
    assert sorted(written) == sorted(lists.tolist())
    assert len(set(written)) == len(written) and max(written) < npart
    assert (np.diff(tiles[:, 4]) == tiles[:-1, 5]).all()     # CSR offsets
    for t in tiles:
        seg = lists[t[4]:t[4] + t[5]]
        assert (np.diff(seg) > 0).all()                      # unit order = increasing index


@pytest.mark.parametrize("n_h,n_e", CASES)
def test_update_units_follow_their_slots_pair_units(lib, n_h, n_e):
    rc, units, tiles, lists, npart = cts.cts_plan_sym(n_h, n_e)
    assert rc == 0
    for s, (nh, ne) in enumerate(zip(n_h, n_e)):
        pos = np.flatnonzero(units[:, 0] == s)
        kinds = units[pos, 10]
        if nh <= 0:
            assert len(pos) == 0
            continue
        nt = _tiles_of(nh) + _tiles_of(ne)
        pair_pos, upd_pos = pos[kinds == 0], pos[kinds == 1]
        assert pair_pos.max() < upd_pos.min()          # every pair unit earlier in the queue
        assert (units[upd_pos, 11] == len(pair_pos)).all()
        cover = np.zeros(nt, dtype=int)
        for u in units[upd_pos]:
            assert u[6] - u[5] == max(1, -(-nt // 64)) or u[6] == nt
            cover[u[5]:u[6]] += 1
        assert (cover == 1).all()                      # each tile updated once
        assert len(upd_pos) <= 64


def test_symmetric_plan_unit_shapes_and_limits(lib):
    # small events: 1 block x 8 tiles; larger: 2 x 16; largest: 8 x 16
    for n, (rb, rj) in [(5525, (1, 8)), (20000, (2, 16)), (50000, (8, 16))]:
        rc, units, *_ = cts.cts_plan_sym([n], [0])
        assert rc == 0
        units = _pairs(units)
        assert (units[:, 4] - units[:, 3]).max() == rb
        assert (units[:, 6] - units[:, 5]).max() == rj
    # too many units for the buffer
    rc, *_ = cts.cts_plan_sym([5525] * 64, [0] * 64, max_units=100)
    assert rc == -2
    # a finished event (no holes) gets nothing
    rc, units, tiles, lists, npart = cts.cts_plan_sym([0, 0], [10, 0])
    assert rc == 0 and len(units) == 0 and len(tiles) == 0 and npart == 0


def _emulate_field(xyz, n_h, n_e, eps):
    """The kernel's arithmetic in FP64 numpy on the plan of one slot: units
    write s_j * sum d w (I partials) and -s_i * sum d w (J partials), d = r_i -
    r_j, w = (|d|^2 + eps^2)^-1.5; a tile's field is the sum of its list."""
    rc, units, tiles, lists, npart = cts.cts_plan_sym([n_h], [n_e])
    assert rc == 0
    part = np.zeros((npart, 3, T))
    rng = {0: (0, n_h), 1: (n_h, n_h + n_e)}
    sgn = {0: 1.0, 1: -1.0}

    def tile_pos(spec, t):
        a, b = rng[spec]
        idx = np.arange(a + t * T, min(a + (t + 1) * T, b))
        return idx

    for u in _pairs(units):
        _, si, sj, ib0, ib1, jt0, jt1, pi, pj = (int(v) for v in u[:9])
        nti = _tiles_of(n_e if si else n_h)
        isum = {}
        jsum = {g: np.zeros((3, T)) for g in range(jt0, jt1)}
        for ti, tj, mode in _combos(u, nti):
            ii, jj = tile_pos(si, ti), tile_pos(sj, tj)
            d = xyz[ii][:, None, :] - xyz[jj][None, :, :]
            w = ((d ** 2).sum(-1) + eps * eps) ** -1.5
            t = d * w[..., None]                          # [i, j, 3]
            acc = isum.setdefault(ti, np.zeros((3, T)))
            acc[:, :len(ii)] += t.sum(1).T
            if mode == 2:
                jsum[tj][:, :len(jj)] += t.sum(0).T
        for b in range(ib0, ib1):
            for q in range(TPB):
                if b * TPB + q < nti:
                    part[pi + (b - ib0) * TPB + q] = sgn[sj] * isum.get(b * TPB + q, 0.0)
        for g in range(jt0, jt1):
            part[pj + g - jt0] = -sgn[si] * jsum[g]
    E = np.zeros((n_h + n_e, 3))
    th = _tiles_of(n_h)
    for k, t in enumerate(tiles):
        spec, tile, n = int(t[1]), int(t[2]), int(t[3])
        f = part[lists[t[4]:t[4] + t[5]]].sum(0)          # [3, T]
        idx = tile_pos(spec, tile)
        assert len(idx) == n and k == (th if spec else 0) + tile
        E[idx] = f[:, :n].T
    return E


@pytest.mark.parametrize("n_h,n_e", [(300, 0), (257, 3), (130, 70), (64, 64), (1, 0), (2, 1),
                                     (700, 450)])
def test_symmetric_emulation_matches_the_oracle_field(n_h, n_e):
    oracle.build()
    rng = np.random.default_rng(n_h * 1000 + n_e)
    xyz = np.concatenate([rng.standard_normal((n_h, 3)),
                          rng.standard_normal((n_e, 3)) + [0.4, 0.0, 0.5]])
    eps = 1e-6
    sign = np.r_[np.ones(n_h), -np.ones(n_e)].astype(np.int8)
    ref = oracle.field(xyz, sign=sign, kc=1.0, eps=eps)
    got = _emulate_field(xyz, n_h, n_e, eps)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
