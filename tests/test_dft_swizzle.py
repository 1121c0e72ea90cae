"""Host enumeration of the shared-memory layout of the n = 2048 forward DFT kernel that
loads its rings by bulk copies (k_fft_fwd_sw in fft32.cu): point i of a ring sits at
swz(i) = i ^ ((i >> 4) & 7) ^ (((i >> 7) & 1) << 3) once the first stage has run.  For every
warp-wide 8-byte access of the kernel's stages, each half-warp must touch 16 distinct
slots (address mod 16 complexes), i.e. the minimum of two wavefronts per warp; the first
stage's writes must stay inside the 16-point groups its warp read; the map must be a
permutation.  The records' negative-order bins may take up to twice that, as in the
padded layout of the other kernels.  swz is restated here from the kernel's definition."""
N = 2048


def swz(a):
    return a ^ ((a >> 4) & 7) ^ (((a >> 7) & 1) << 3)


def wavefronts(addrs):
    tot = 0
    for h in range(2):
        slots = {}
        for a in set(addrs[16 * h:16 * h + 16]):
            slots.setdefault(a % 16, set()).add(a)
        tot += max(len(v) for v in slots.values())
    return tot


def nib(b):
    return ((b & 15) << 4) | (b >> 4)


def test_permutation_within_groups():
    assert sorted(swz(a) for a in range(4 * N)) == list(range(4 * N))
    assert all(swz(a) >> 4 == a >> 4 for a in range(4 * N))


def test_stage_accesses_conflict_free():
    for warp in range(16):
        ts = [warp * 32 + l for l in range(32)]
        for q in range(16):
            assert wavefronts([(t >> 7) * N + (t & 127) + 128 * q for t in ts]) == 2
            assert wavefronts([swz((t >> 7) * N + (t & 127) + 128 * q) for t in ts]) == 2
            assert wavefronts([swz((t >> 7) * N + ((t & 127) >> 3) * 128 + (t & 7) + 8 * q) for t in ts]) == 2
        for u in range(2):
            idx = [t % 256 + 512 * u + 256 * (t // 256) for t in ts]
            for q in range(8):
                assert wavefronts([swz((i >> 8) * N + (i & 255) * 8 + q) for i in idx]) == 2
                assert wavefronts([swz((i >> 8) * N + nib(i & 255) + 256 * q) for i in idx]) == 2


def test_record_bins():
    for mu0 in range(0, 1024, 32):
        for c in range(4):
            assert wavefronts([swz(c * N + mu0 + l) for l in range(32)]) == 2
            assert wavefronts([swz(c * N + ((N - mu0 - l) if mu0 + l else 0)) for l in range(32)]) <= 4


def quarter_wavefronts(addrs16):
    """16-byte accesses: per quarter-warp, the largest number of distinct addresses that share
    one of the 8 16-byte bank groups."""
    tot = 0
    for qw in range(4):
        groups = {}
        for a in set(addrs16[8 * qw:8 * qw + 8]):
            groups.setdefault(a % 8, set()).add(a)
        tot += max(len(v) for v in groups.values())
    return tot


def ring_base(r):
    """k_fft_inv_sw: ring r shifted by 8 r complexes (the rings do not overlap)."""
    return r * (N + 8)


def test_inverse_rings_disjoint():
    spans = [(ring_base(r), ring_base(r) + N) for r in range(4)]
    assert all(spans[r][1] <= spans[r + 1][0] for r in range(3)) and spans[3][1] <= 4 * N + 24


def test_inverse_record_reads_and_bin_writes():
    # a thread takes component tsk & 1 of order tsk >> 1 of a 256-order box; the box holds
    # [order][parity][2 components][4 floats] (16-byte units), read parity p0 first, p0 = (r >> 1) & 1
    for w in range(8):
        tsk = [32 * w + l for l in range(32)]
        for step in range(2):
            addrs = []
            for t in tsk:
                r, comp = t >> 1, t & 1
                p0 = (r >> 1) & 1
                addrs.append(r * 4 + (p0 ^ step) * 2 + comp)
            assert quarter_wavefronts(addrs) == 4
    # the bins +mu of rings comp and 2 + comp (8-byte writes)
    for box in range(4):
        for w in range(8):
            for it in range(2):
                lanes = [it * 256 + 32 * w + l for l in range(32)]
                for rr in (0, 2):
                    plus = [ring_base(rr + (t & 1)) + swz(box * 256 + (t >> 1)) for t in lanes]
                    assert wavefronts(plus) == 2
                    mus = [box * 256 + (t >> 1) for t in lanes]
                    minus = [ring_base(rr + (t & 1)) + swz(N - mu) for t, mu in zip(lanes, mus) if mu]
                    assert wavefronts(minus + [minus[-1]] * (32 - len(minus))) <= 4
