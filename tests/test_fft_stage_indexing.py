"""Host check of the compile-time Stockham stage's index arithmetic
(fft_stage_ct in csrc/dgpe_device.cuh), replayed in Python for every
(length, elements per thread, lines, threads) the kernels instantiate: each
stage's reads and writes stay inside the tile and touch every element of every
line exactly once, and the radix sequence matches the runtime plans' order
(16, 8, 5, 4, 3, 2).  A stage that took a thread's butterfly slots as all real
whenever the butterfly count was a multiple of the block size read past the
tile for 96 and 384 (12 elements per thread); the replay of that condition
fails here."""
import pytest


def ct_radix(n, ept, s):
    m = n
    for k in range(16):
        r = 0
        for c in (16, 8, 5, 4, 3):
            if ept % c == 0 and m % c == 0:
                r = c
                break
        if r == 0 and m % 2 == 0:
            r = 2
        if r == 0:
            return 0
        if k == s:
            return r
        m //= r
    return 0


def nstages(n, ept):
    s, m = 0, n
    while m > 1:
        m //= ct_radix(n, ept, s)
        s += 1
    return s


def replay(N, EPT, NL, T, line_fast, inv, full=lambda B, T, NB: B == T * NB):
    NS, S = 1, nstages(N, EPT)
    for s in range(S):
        RAD = ct_radix(N, EPT, S - 1 - s if inv else s)
        NB, NBL = EPT // RAD, N // RAD
        B = NBL * NL
        assert B <= T * NB
        reads, writes = set(), set()
        for t in range(T):
            for i in range(NB):
                b = t + i * T
                if not (full(B, T, NB) or b < B):
                    continue
                l, j = (b % NL, b // NL) if line_fast else (b // NBL, b % NBL)
                assert l < NL and j < NBL
                for r in range(RAD):
                    a = j + r * NBL
                    assert a < N and (l, a) not in reads
                    reads.add((l, a))
                base = (j // NS) * NS * RAD + j % NS
                for r in range(RAD):
                    a = base + r * NS
                    assert a < N and (l, a) not in writes
                    writes.add((l, a))
        assert len(reads) == len(writes) == N * NL
        NS *= RAD


CASES = ([(N, 8, 128 // (N // 16), 256, False) for N in (32, 64, 128, 256, 512)]
         + [(N, 12, 128 // (N // 12), 256, False) for N in (96, 192, 384)]
         + [(N, 20, 128 // (N // 10), 256, False) for N in (160, 320)]
         + [(64, 8, 32, 256, False)]
         + [(N, 16, 256 * 16 // N, 256, True) for N in (64, 128, 256, 512)]
         + [(N, 12, 256 * 12 // N, 256, True) for N in (96, 384)]
         + [(160, 20, 32, 256, True)]
         + [(N, 16, W, W * N // 16, True) for W in (16, 8, 4) for N in (32, 64, 128, 256, 512)
            if W * N // 16 <= 256])


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("inv", [False, True])
def test_stage_indices_in_bounds_and_exact(case, inv):
    replay(*case, inv=inv)


def test_radix_order_matches_runtime_plans():
    assert [ct_radix(384, 12, s) for s in range(nstages(384, 12))] == [4, 4, 4, 3, 2]
    assert [ct_radix(160, 20, s) for s in range(nstages(160, 20))] == [5, 4, 4, 2]
    assert [ct_radix(256, 8, s) for s in range(nstages(256, 8))] == [8, 8, 4]


def test_old_coverage_condition_fails():
    with pytest.raises(AssertionError):
        replay(96, 12, 16, 256, False, False, full=lambda B, T, NB: B % T == 0)
