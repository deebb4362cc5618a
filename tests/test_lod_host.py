"""Host logic of the ranked LoD (CPU): nested prefix orders and template
permutation."""
import math

import numpy as np

from paper_2501_17792_gb300 import lod as LOD
from paper_2501_17792_gb300 import scene as S


def test_prefix_orders_are_nested_top_sets():
    rng = np.random.default_rng(3)
    sizes = [500, 333]
    scores = rng.normal(size=(3, sum(sizes)))
    fr = [1.0, 0.3, 0.07]
    orders = LOD.prefix_orders(scores, fr, sizes)
    off = 0
    for n, o in zip(sizes, orders):
        assert sorted(o.tolist()) == list(range(n))  # a permutation
        s = scores[:, off:off + n]
        n2 = int(math.floor(fr[2] * n + 0.5))
        n1 = int(math.floor(fr[1] * n + 0.5))
        # the coarsest level is exactly that band's top set
        assert set(o[:n2].tolist()) == set(np.argsort(-s[2])[:n2].tolist())
        # the next level adds the best of band 1 among the rest
        rest = np.setdiff1d(np.arange(n), o[:n2])
        want = rest[np.argsort(-s[1, rest], kind="stable")[:n1 - n2]]
        assert set(o[n2:n1].tolist()) == set(want.tolist())
        off += n


def test_permute_template_reorders_every_per_gaussian_array():
    t = S.make_template(5, 64, 1)
    perm = np.random.default_rng(1).permutation(64)
    p = LOD.permute_template(t, perm)
    for name in ("means", "scales", "quats", "opacity", "sh", "skin_idx", "skin_w"):
        assert np.array_equal(getattr(p, name), getattr(t, name)[perm]), name
    assert np.array_equal(p.rest_joints, t.rest_joints) and np.array_equal(p.parents, t.parents)
