"""The allocation-free entry point (vafr_morton_sort_noalloc), for callers that
may not allocate device memory -- e.g. code whose GPU memory all belongs to its
own pool allocator, or a latency-critical thread that must not take
cudaMalloc's implicit synchronisation.  Its Morton codes and sorted order must
equal what vafr_build_scene computes (integer results: bit-exact), on two calls
in a row that share the one scratch array.  Collected last on purpose."""

import numpy as np
import pytest

from workloads import random_triangles_scene, terrain_boxes_scene

pytestmark = pytest.mark.gpu


def _reference(V, torch, tris):
    h = V.vafr_build_scene(tris, None, (0.0, -1.0, 0.0))
    codes, ids, _, _, _ = V.vafr_scene_export_lbvh(h)
    V.vafr_scene_destroy(h)
    return codes, ids


def _noalloc(V, torch, tris):
    n = tris.shape[0]
    codes = torch.empty(n, dtype=torch.int32, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    V.vafr_morton_sort_noalloc(tris, codes, ids)
    torch.cuda.synchronize()
    return codes.cpu().numpy().view(np.uint32), ids.cpu().numpy()


def test_noalloc_matches_build_on_two_calls_in_a_row(V, torch_mod):
    torch = torch_mod
    big = terrain_boxes_scene(256, 1024, 300, seed=31).tris      # 525,618 tris: too many
    a = torch.from_numpy(np.ascontiguousarray(big[:500_000].reshape(-1, 9))).cuda()
    b = torch.from_numpy(np.ascontiguousarray(random_triangles_scene(33_333, seed=5).tris.reshape(-1, 9))).cuda()
    for tris in (a, b):            # the second, smaller call follows the first in the same scratch
        codes, ids = _noalloc(V, torch, tris)
        rc, rid = _reference(V, torch, tris)
        assert np.array_equal(codes, rc)
        assert np.array_equal(ids, rid)


def test_noalloc_rejects_oversized_and_host_input(V, torch_mod):
    torch = torch_mod
    n = V.NOALLOC_MAX_TRIS + 1
    tris = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VafrError, match="VAFR_NOALLOC_MAX_TRIS"):
        V.vafr_morton_sort_noalloc(tris, out, out)
    host = np.zeros((8, 9), np.float32)
    small = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VafrError, match="device memory"):
        V.vafr_morton_sort_noalloc(host, small, small)


def test_noalloc_rejects_overlapping_buffers(V, torch_mod):
    """Outputs that share bytes with each other or with the input would corrupt
    the sort silently; the entry point refuses them before any launch."""
    torch = torch_mod
    n = 1000
    tris = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    out = torch.empty(3 * n, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VafrError, match="overlap"):
        V.vafr_morton_sort_noalloc(tris, out[:n], out[n // 2:n // 2 + n])      # outputs overlap
    with pytest.raises(V.VafrError, match="overlap"):
        V.vafr_morton_sort_noalloc(tris, tris.view(torch.int32).view(-1)[:n], out[:n])   # code over input
    V.vafr_morton_sort_noalloc(tris, out[:n], out[n:2 * n])                      # adjacent: fine
    torch.cuda.synchronize()
