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


def test_checkpoint_blocks_cover_the_run_with_the_full_block_last():
    from paper_1906_10811_b300.fwi import blocks
    for nt in (1, 5, 60, 70, 1000):
        for k in (1, 3, 7, 9, 25, 60, 975, 1000):
            if k > nt:
                continue
            b = blocks(nt, k)
            assert len(b) == -(-nt // k)
            assert b[0][0] == 0 and b[-1][1] == nt
            assert all(b[i][1] == b[i + 1][0] for i in range(len(b) - 1))
            assert all(0 < n1 - n0 <= k for n0, n1 in b)
            assert b[-1][1] - b[-1][0] == k          # the forward sweep's own block is full
            assert all(n1 - n0 == k for n0, n1 in b[1:])
