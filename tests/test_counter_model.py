"""The carry-save counters of the threshold kernels as arithmetic (no GPU): S
bit slices plus a sticky slice, inputs added four at a time through full
adders (sum = XOR3, carry = MAJ3) with the weight-2^S carry ORed into the
sticky slice, then the bit-sliced compare "count >= thr" for 1 <= thr <= 2^S
(thr = 2^S is the sticky slice alone).  Restated here over 32-bit words and
checked against per-row counts: every threshold up to 2^S is decided
exactly, which is why S = ceil(log2 T) slices suffice for a threshold T."""
import numpy as np
import pytest

M32 = 0xFFFFFFFF


class Counters:
    def __init__(self, S):
        self.S = S
        self.c = [0] * S
        self.sticky = 0

    def _add1(self, K, x):
        for j in range(K, self.S):
            t = self.c[j] & x
            self.c[j] ^= x
            x = t
        self.sticky |= x

    def _add2(self, K, x, y):
        if K < self.S:
            a = self.c[K]
            self.c[K] = a ^ x ^ y
            return (a & x) | (a & y) | (x & y)
        self.sticky |= x | y
        return 0

    def add4(self, a, b, c, d):
        k1 = self._add2(0, a, b)
        k2 = self._add2(0, c, d)
        k3 = self._add2(1, k1, k2)
        if self.S > 2:
            self._add1(2, k3)
        else:
            self.sticky |= k3

    def ge(self, thr):
        if thr >> self.S:
            return self.sticky
        eq, gt = M32, 0
        for k in range(self.S - 1, -1, -1):
            if (thr >> k) & 1:
                eq &= self.c[k]
            else:
                gt |= eq & self.c[k]
                eq &= ~self.c[k] & M32
        return gt | eq | self.sticky


def slices_for(t):
    return 1 if t <= 2 else int(t - 1).bit_length()


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_every_threshold_up_to_two_to_the_s(S):
    rng = np.random.default_rng(S)
    for trial in range(40):
        n = int(rng.integers(1, 4 * (1 << S) + 8))
        p = float(rng.uniform(0.02, 0.9))
        x = (rng.random((n, 32)) < p).astype(np.int64)
        words = [int(sum(int(b) << i for i, b in enumerate(row))) for row in x]
        while len(words) % 4:
            words.append(0)  # absent inputs of a group are zero words
        cnt = Counters(S)
        for i in range(0, len(words), 4):
            cnt.add4(*words[i:i + 4])
        count = x.sum(axis=0)
        for thr in range(1, (1 << S) + 1):
            got = cnt.ge(thr)
            want = sum(1 << i for i in range(32) if count[i] >= thr)
            assert got == want, (S, n, thr)
        # the lowest slice is the parity of the count
        assert cnt.c[0] == sum(1 << i for i in range(32) if count[i] % 2)


def test_slices_for_is_the_least_width_with_two_to_the_s_at_least_t():
    for t in range(1, 70000, 7):
        s = slices_for(t)
        assert (1 << s) >= t and (s == 1 or (1 << (s - 1)) < t)
