"""Bit-exact parity at the benchmark configurations' own shapes.

Every level of the trees the benchmark builds -- bitmap words, rank
directory R and Hy, select samples S1 and S0, ones count -- equals the CPU
oracle's, element by element:
  * the text (2^30 bytes over 96 codes, Zipf 1.0), DNA (2^30 bytes over 4
    codes) and word (2^29 four-byte codes over 2^20, Zipf 1.2) sequences,
    built as bench.py builds them (wt_build_async, automatic variant); the
    oracle computes each level alone by Algorithm 1's per-level body, one
    level per host core;
  * the batch of 4096 sequences (lengths log-uniform in [2^10, 2^22],
    alphabets {4, 20, 256, 65536}, uniform or Zipf 1.1), built by one
    wt_build_batch call as bench.py builds it; every sequence's oracle tree
    is computed on the host cores and each level is compared through a
    digest of all its arrays, with an element-by-element diff of any level
    whose digest differs.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, wt
from oracle import oracle as O
from oracle_pool import batch_digests, level_digest, tree_levels
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow, needs_gpu]


def _first_diff(got: np.ndarray, want: np.ndarray) -> str:
    if got.shape != want.shape:
        return f"shape {got.shape} != {want.shape}"
    bad = np.flatnonzero(got != want)
    return f"{len(bad)} elements differ, first at {bad[0]}"


@pytest.mark.parametrize("name", ["u8-text-2^30-s96-zipf1.0", "u8-dna-2^30-s4", "u32-words-2^29-s2^20-zipf1.2"])
def test_full_size_every_level_bit_exact(name):
    W = wt()
    w = inputs.WORKLOADS[name]
    S = w.generate()
    dev = torch.from_numpy(S).cuda()
    tree = W.Tree.build(dev, w.sigma, wait=False)
    tree.wait()
    del dev
    seen = set()
    for l, bits, d in tree_levels(S, w.sigma):
        lv = tree.level(l)
        got = lv.words.cpu().numpy().view(np.uint8)
        assert np.array_equal(got, bits), f"{name} level {l} bitmap: {_first_diff(got, bits)}"
        for key, arr in (("R", lv.R), ("Hy", lv.Hy), ("S1", lv.S1), ("S0", lv.S0)):
            g = arr.cpu().numpy()
            assert np.array_equal(g, d[key]), f"{name} level {l} {key}: {_first_diff(g, d[key])}"
        assert lv.ones == d["ones"], f"{name} level {l} ones"
        seen.add(l)
        del lv, got
    assert seen == set(range(O.levels(w.sigma)))
    tree.free()
    torch.cuda.empty_cache()


def test_batch_at_its_configuration_shape_bit_exact():
    """4096 sequences in one wt_build_batch call on a side stream, packed in
    one device buffer at 256-byte aligned starts, exactly as bench.py's
    batched workload builds them."""
    W = wt()
    specs = inputs.batch_specs(4096)
    want = batch_digests(specs)
    host = [sp.generate() for sp in specs]
    offs, total = [], 0
    for h in host:
        offs.append(total)
        total += (h.nbytes + 255) // 256 * 256
    stage = np.zeros(total, np.uint8)
    for h, o in zip(host, offs):
        stage[o:o + h.nbytes] = h.view(np.uint8)
    buf = torch.from_numpy(stage).cuda()
    tdt = {1: torch.uint8, 2: torch.uint16}
    seqs = [buf[o:o + h.nbytes].view(tdt[h.itemsize]) for h, o in zip(host, offs)]
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    trees = W.build_batch(seqs, [sp.sigma for sp in specs], stream=st, wait=False)
    for t in trees:
        t.wait()
    bad = []
    for k, (sp, t) in enumerate(zip(specs, trees)):
        for l, wd in enumerate(want[k]):
            lv = t.level(l)
            got = level_digest(lv.words.cpu().numpy().view(np.uint8), lv.R.cpu().numpy(), lv.Hy.cpu().numpy(),
                               lv.S1.cpu().numpy(), lv.S0.cpu().numpy(), lv.ones)
            if got != wd:
                bad.append((k, l))
    if bad:
        k, l = bad[0]
        compare_tree(trees[k], host[k], specs[k].sigma)   # raises with the first differing element
        raise AssertionError(f"{len(bad)} levels differ, first sequence {k} level {l}")
    assert sum(len(d) for d in want) == sum(O.levels(sp.sigma) for sp in specs)
    for t in trees:
        t.free()
    del buf, seqs
    torch.cuda.empty_cache()
