"""GPU test of the tree compression's CUDA graphs (ffc_params.graphs): every sample-size round is captured
into a graph the first time it runs on a result and replayed as one graph launch when it recurs. The
graphs hold the same memsets and launches as the direct form, so every output is bitwise identical, and
a second call on the same tree captures nothing new. The profile's phase events are graph nodes, so
the phase times stay available."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")
KEYS = ("node", "rank", "s", "status", "r22_rel", "log_scale", "far_count", "rows", "skel", "T", "ncols", "cols")


def _tree(N, d, seed):
    P = workloads.gaussian_mixture(N=N, d=d, k=4, seed=seed)
    t = ffc.ffc_build_tree(torch.tensor(P, device=DEV), 256)
    return torch.tensor(P, device=DEV)[t.perm].contiguous(), t


def _same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("d,kind,nested", [(16, ffc.GAUSSIAN, False), (128, ffc.POLYNOMIAL, False),
                                           (16, ffc.GAUSSIAN, True)])
def test_graph_rounds_match_direct_launches_and_replay(d, kind, nested):
    Pp, t = _tree(16384, d, seed=d)
    k = ffc.Kernel(kind, h=2.0) if kind == ffc.GAUSSIAN else ffc.Kernel(kind, h=float(d), c=1.0, p=3)
    kw = dict(tol=1e-6, precision=ffc.MIXED, s0=128, s_max=1024, nested=nested)
    direct = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t, k, graphs=False, **kw))
    res = ffc.ffc_compress_tree(Pp, t, k, **kw)
    _same(ffc.tree_result_to_host(res), direct)
    res.profile_enable(True)      # the phase events join the graphs: every round is captured once more
    res.profile_reset()
    res = ffc.ffc_compress_tree(Pp, t, k, result=res, **kw)
    p1 = res.profile()
    assert p1["graph_captures"] == p1["rounds"] >= 2 and p1["graph_launches"] == p1["rounds"]
    _same(ffc.tree_result_to_host(res), direct)
    res = ffc.ffc_compress_tree(Pp, t, k, result=res, **kw)
    p2 = res.profile()
    assert p2["graph_captures"] == p1["graph_captures"]            # every round replayed
    assert p2["graph_launches"] == 2 * p1["graph_launches"]
    assert all(v > 0 for v in p2["ms"].values())
    _same(ffc.tree_result_to_host(res), direct)


def test_graphs_with_the_learned_sampler_match_direct_launches():
    Pp, t = _tree(16384, 16, seed=3)
    k = ffc.Kernel(ffc.GAUSSIAN, h=2.0)
    params = torch.tensor(workloads.mlp_init(4).astype(np.float32), device=DEV)
    proj = torch.as_tensor(workloads.projections(16, seed=7)).to(DEV)
    kw = dict(tol=1e-6, precision=ffc.MIXED, s0=128, s_max=1024, proposal=(params, proj))
    direct = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t, k, graphs=False, **kw))
    res = ffc.ffc_compress_tree(Pp, t, k, **kw)
    res = ffc.ffc_compress_tree(Pp, t, k, result=res, **kw)
    _same(ffc.tree_result_to_host(res), direct)
