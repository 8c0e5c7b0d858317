"""Host-side plans of the simulated collectives (CPU only): the library's
chunk partition and recursive-doubling schedule agree with the oracle's, so
the GPU ranks and the oracle ranks reduce the same chunks in the same order."""
from paper_2308_05199_gb300 import collectives as C

import oracle


def test_chunk_partition_matches_the_oracle():
    for P in range(1, 10):
        for n in list(range(0, 40)) + [1000, 1 << 20, (1 << 26) + 7]:
            b = C.chunk_bounds(n, P)
            assert b == oracle.chunk_bounds(n, P)
            assert b[0] == 0 and b[-1] == n and len(b) == P + 1
            sizes = [b[c + 1] - b[c] for c in range(P)]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_recursive_doubling_schedule_matches_the_oracle():
    for N in range(1, 70):
        k, r, active = C.redoub_plan(N)
        assert (k, r, active) == oracle.redoub_plan(N)
        assert (1 << k) <= N < (1 << (k + 1)) and r == N - (1 << k)
        assert len(active) == 1 << k and len(set(active)) == len(active)
        folded = [i for i in range(2 * r) if i % 2 == 0]
        assert set(active) | set(folded) == set(range(N))
