"""Host logic of the FWI driver (no GPU): checkpoint memory and the tuner's candidates."""


def test_checkpoint_candidates_and_memory():
    """Host logic of the checkpoint tuner: memory formula and candidate list."""
    from paper_1906_10811_b300 import fwi
    assert fwi.checkpoint_memory(1000, 1000, 1) == 1000 + 2 + 2
    assert fwi.checkpoint_memory(1000, 45, 1) == 45 + 2 + 2 * 23
    c = fwi.checkpoint_candidates(1000, 1, 10 ** 6)
    assert c[0] == min(range(1, 1001), key=lambda k: (fwi.checkpoint_memory(1000, k, 1), k))
    assert 40 <= c[0] <= 50 and c[-1] == 1000 and c == sorted(set(c))
    tight = fwi.checkpoint_candidates(1000, 1, 200)
    assert all(fwi.checkpoint_memory(1000, k, 1) <= 200 for k in tight)
