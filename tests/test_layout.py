"""Host logic of the work decomposition (ss_layout, ss_layout_warps; no GPU): the S3
tiles of K2 (64 x 64 tiles, or the 32 x 32 sub-tiles of the independent-warp form)
and the points left to the point kernel cover the bispectrum domain (Eq. 28 / Eq. 48)
exactly once; the tensor-core S4 tiles and the column left to the column kernel
cover the upper triangle k <= l of the trispectrum cut exactly once."""
import numpy as np
import pytest

TS = [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


def P():
    import paper_2505_01231_gb300 as mod
    return mod


def dom3(k, l, M, cross):
    if cross:
        return 0 <= l < M and -M < k < M and -M < k + l < M
    return 0 <= k <= l and k + l < M


@pytest.mark.parametrize("channels", [1, 2])
@pytest.mark.parametrize("T", TS)
def test_s3_tiles_and_points_cover_the_domain_once(T, channels):
    mod = P()
    M = T // 2 + 1
    cross = channels > 1
    t3, pts, _, _ = mod.ss_layout(channels, T)
    k = np.arange(-(M - 1), M)[:, None]
    l = np.arange(M)[None, :]
    want = (l >= 0) & (l < M) & (np.abs(k + l) <= M - 1) if cross else \
        (k >= 0) & (k <= l) & (k + l < M)
    cover = np.zeros(want.shape, int)
    for k0, l0 in t3:
        assert k0 % 64 == 0 and l0 % 64 == 0
        ks = slice(max(k0, -(M - 1)) + M - 1, min(k0 + 64, M) + M - 1)
        ls = slice(l0, min(l0 + 64, M))
        inside = want[ks, ls].sum()
        assert inside > (0 if cross else 8), (k0, l0, inside)
        cover[ks, ls] += want[ks, ls]
    if cross:
        assert pts == []
    for kp, lp in pts:
        assert dom3(kp, lp, M, cross)
        cover[kp + M - 1, lp] += 1
    assert np.array_equal(cover, want.astype(int))


@pytest.mark.parametrize("T", TS)
def test_independent_warp_subtiles_and_points_cover_the_domain_once(T):
    mod = P()
    M = T // 2 + 1
    tiles, pts = mod.ss_layout_warps(T)
    k = np.arange(M)[:, None]
    l = np.arange(M)[None, :]
    want = ((k <= l) & (k + l < M)).astype(int)
    cover = np.zeros((M, M), int)
    for k0, l0 in tiles:
        assert k0 % 32 == 0 and l0 % 32 == 0 and 0 <= k0 < M and 0 <= l0 < M
        inside = want[k0:k0 + 32, l0:l0 + 32]
        assert inside.sum() > 8, (k0, l0)
        cover[k0:k0 + 32, l0:l0 + 32] += inside
    for kp, lp in pts:
        assert dom3(kp, lp, M, False)
        # a point of the list lies in a sub-tile with at most 8 domain points
        k0, l0 = kp // 32 * 32, lp // 32 * 32
        assert want[k0:k0 + 32, l0:l0 + 32].sum() <= 8 and (k0, l0) not in tiles
        cover[kp, lp] += 1
    assert np.array_equal(cover, want)


def test_layout_warps_rejects_bad_shapes():
    mod = P()
    for T in (4, 100, 8192):
        with pytest.raises(mod.SSError) as ei:
            mod.ss_layout_warps(T)
        assert ei.value.status == mod.SS_EINVAL


@pytest.mark.parametrize("T", TS)
def test_tensor_core_tiles_and_column_cover_the_triangle_once(T):
    mod = P()
    M = T // 2 + 1
    _, _, t4, col = mod.ss_layout(1, T)
    k = np.arange(M)[:, None]
    l = np.arange(M)[None, :]
    want = (k <= l).astype(int)
    cover = np.zeros((M, M), int)
    for k0, l0, n in t4:
        assert k0 % 128 == 0 and l0 % 128 == 0 and n % 16 == 0 and 16 <= n <= 128
        cover[k0:min(k0 + 128, M), l0:min(l0 + n, M)] += want[k0:min(k0 + 128, M),
                                                             l0:min(l0 + n, M)]
    assert col == ((M - 1) % 128 == 0 and M > 1)
    if col:
        cover[:, M - 1] += want[:, M - 1]
    assert np.array_equal(cover, want)


def test_layout_rejects_bad_shapes():
    mod = P()
    for channels, T in ((0, 64), (5, 64), (1, 100), (1, 4), (1, 8192)):
        with pytest.raises(mod.SSError) as ei:
            mod.ss_layout(channels, T)
        assert ei.value.status == mod.SS_EINVAL
