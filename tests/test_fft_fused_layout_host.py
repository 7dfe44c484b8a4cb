"""Host model of the fused-unpack padded FFT's data layout (the kernel
`k_fft_real_fused<LZ, R>`): the staging slots, the fused last Stockham pass
and the unpack, replayed in numpy with the kernel's own index arithmetic.

The padded real FFT (Section 2.1, Eq. 2-3) packs sample pairs into H =
N_FFT/2 complex points z, splits the H-point DFT into R pre-twiddled LZ-point
residue DFTs, and unpacks X[k], X[H - k] from Z[k], Z[H - k].  The kernel runs
the first two radix-16 passes of each residue DFT, stages their outputs at
slot fsw(pos R + r), and each unpack thread computes the rho-point butterflies
of the last pass whose outputs it unpacks.  This test rebuilds that schedule:
every output bin must be written exactly once and equal numpy's FFT, and the
shared-memory accesses the swizzle is meant to keep conflict-free must be so.
No GPU: it pins the layout the kernel was written from."""
import numpy as np
import pytest

TWO_PI = 2 * np.pi


def w(num, den):
    return np.exp(-1j * TWO_PI * (num % den) / den)


def wpi32(a):
    return np.exp(-1j * np.pi * a / 32)


def fsw(x):
    """Staging slot of x (float2 units): the 16-byte chunk index within each
    128-byte row XORed with the row index mod 8."""
    return x ^ (((x >> 4) & 7) << 1)


def residue_partials(z, r, H, LZ, rho):
    """Outputs of the first two passes of residue r in Stockham order: the
    NS-point DFTs of the decimated, pre-twiddled input, a[j + m NS].  A z
    longer than LZ is folded first: z[m0] + z[m0 + LZ] w_R^r (R = H/LZ)."""
    NS = LZ // rho
    if len(z) > LZ:
        z = z[:LZ] + z[LZ:] * w(r, H // LZ)
    v = z * w(r * np.arange(LZ), H)
    a = np.zeros(LZ, complex)
    for m in range(rho):
        a[m * NS:(m + 1) * NS] = np.fft.fft(v[m::rho])
    return a


def bank_ways(words, width):
    """Largest number of distinct 32-bit words one bank serves for accesses
    starting at `words` (each `width` words wide)."""
    banks = {}
    for a in words:
        for d in range(width):
            banks.setdefault((a + d) % 32, set()).add(a + d)
    return max(len(v) for v in banks.values())


def fused_model(LZ, R, seed, plant=None, fold=1):
    H = R * LZ
    rho = 1 << (int(np.log2(LZ)) % 4)
    NS, HB, J = LZ // rho, H // rho, 16 // rho
    T, G = LZ // 16, R // 2
    PT = G * T
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(2 * LZ * fold)
    z = x[0::2] + 1j * x[1::2]
    parts = {r: residue_partials(z, r, H, LZ, rho) for r in range(R)}

    # staging: thread (pair gl, t) holds pass-1 output r at pos0 + 16 r for
    # residues 2 gl and 2 gl + 1 and stores them as one 16-byte pair
    stage = np.full(H, np.nan + 0j)
    for gl in range(G):
        for t in range(T):
            pos0 = (t - (t & 15)) * 16 + (t & 15)
            for r in range(16):
                s = fsw((pos0 + 16 * r) * R + 2 * gl)
                assert s % 2 == 0
                stage[s] = parts[2 * gl][pos0 + 16 * r]
                stage[s + 1] = parts[2 * gl + 1][pos0 + 16 * r]
    assert not np.isnan(stage).any()

    X = np.full(H + 1, np.nan + 0j)
    count = np.zeros(H + 1, int)

    def unpack(k, A, B, wh):                 # wh = w_{2H}^k / 2
        sp, d = 0.5 * (A + np.conj(B)), A - np.conj(B)
        X[k] = sp - 1j * wh * d
        X[H - k] = np.conj(sp + 1j * wh * d)
        count[k] += 1
        count[H - k] += 1

    def butterfly(y, wv):
        y = [y[m] * wv ** m for m in range(rho)]
        return [sum(y[m] * w(m * n, rho) for m in range(rho)) for n in range(rho)]

    for lt in range(PT):
        r, q0 = lt % R, lt // R
        wk0, wq0 = 0.5 * w(lt, 2 * H), w(q0, LZ)
        wm0 = w(NS - 1 - q0 if (r > 0 or plant == "mirror") else NS - q0, LZ)
        zf, zm = fsw(lt), fsw(HB - lt) - HB
        for j in range(J):
            if j == 0 and lt == 0:
                continue
            A = butterfly([stage[zf + PT * j + m * HB] for m in range(rho)], wq0 * wpi32(2 * j))
            B = butterfly([stage[zm + (m + 1) * HB - PT * j] for m in range(rho)], wm0 * np.conj(wpi32(2 * j)))
            k = lt + PT * j
            for n in range(rho):
                tw = wk0 * wpi32(j) * wpi32(32 * n // rho if plant != "twiddle" else 0)
                unpack(k + n * HB, A[n], B[rho - 1 - n], tw)
    # k = 0 and k = HB/2 (residue 0, butterflies 0 and NS/2)
    A = butterfly([stage[fsw(m * HB)] for m in range(rho)], 1.0)
    X[0], X[H] = A[0].real + A[0].imag, A[0].real - A[0].imag
    count[0] += 1
    count[H] += 1
    if rho == 4:
        unpack(HB, A[1], A[3], 0.5 * wpi32(8))
    X[H // 2] = np.conj(A[rho // 2])
    count[H // 2] += 1
    A = butterfly([stage[fsw(HB // 2 + m * HB)] for m in range(rho)], wpi32(32 // rho))
    unpack(HB // 2, A[0], A[rho - 1], 0.5 * wpi32(16 // rho))
    if rho == 4:
        unpack(HB // 2 + HB, A[1], A[2], 0.5 * wpi32(48 // rho))

    # shared-memory banks: staging stores (16 B, 8 lanes per wavefront) and
    # forward reads (8 B, 16 lanes) conflict-free; mirror reads at most 2-way
    worst_st = max(bank_ways([2 * fsw(((t - (t & 15)) * 16 + (t & 15) + 16 * r) * R + 2 * gl)
                              for t in range(t0, t0 + 8)], 4)
                   for gl in range(G) for t0 in range(0, T, 8) for r in range(16))
    worst_f = max(bank_ways([2 * (fsw(lt) + PT * j + m * HB) for lt in range(l0, l0 + 16)], 2)
                  for l0 in range(0, PT, 16) for j in range(J) for m in range(rho))
    worst_m = max(bank_ways([2 * (fsw(HB - lt) - HB + (m + 1) * HB - PT * j) for lt in range(l0, l0 + 16)], 2)
                  for l0 in range(0, PT, 16) for j in range(J) for m in range(rho))
    return x, X, count, (worst_st, worst_f, worst_m)


@pytest.mark.parametrize("LZ,R", [(512, 8), (512, 16), (1024, 4), (1024, 8)])
def test_fused_layout_reproduces_the_padded_fft(LZ, R):
    x, X, count, (st, fwd, mir) = fused_model(LZ, R, seed=LZ + R)
    assert (count == 1).all(), "every bin 0 .. H written exactly once"
    ref = np.fft.rfft(x, 2 * R * LZ)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()
    assert st == 1 and fwd == 1
    assert mir <= 2


@pytest.mark.parametrize("LZ,R", [(512, 8), (512, 16)])
def test_folded_input_reproduces_the_padded_fft(LZ, R):
    # the folded form: traces of 2 LZ sample pairs through LZ-point residues,
    # z[m0] + z[m0 + LZ] w_R^r summed before the pre-twiddle
    x, X, count, _ = fused_model(LZ, R, seed=7 * LZ + R, fold=2)
    assert (count == 1).all()
    ref = np.fft.rfft(x, 2 * R * LZ)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()


def test_planted_fold_twiddle_is_caught():
    # the fold twiddle w_R^r taken with the wrong sign must break the spectrum
    LZ, R = 512, 16
    rng = np.random.default_rng(11)
    z = rng.standard_normal(2 * LZ) + 1j * rng.standard_normal(2 * LZ)
    H = R * LZ
    Z = np.fft.fft(z, H)
    r = 3
    good = np.fft.fft((z[:LZ] + z[LZ:] * w(r, R)) * w(r * np.arange(LZ), H))
    bad = np.fft.fft((z[:LZ] + z[LZ:] * np.conj(w(r, R))) * w(r * np.arange(LZ), H))
    assert np.allclose(good, Z[r::R], rtol=0, atol=1e-9 * np.abs(Z).max())
    assert not np.allclose(bad, Z[r::R], rtol=0, atol=1e-3 * np.abs(Z).max())


@pytest.mark.parametrize("plant", ["mirror", "twiddle"])
def test_planted_index_mistakes_are_caught(plant):
    # the residue-0 mirror butterfly taken by the r > 0 rule, or the unpack
    # twiddle of the outputs k + n H/rho without its e^{-j pi n/rho}: the
    # replayed spectrum must then differ from numpy's
    LZ, R = 512, 8
    x, X, _, _ = fused_model(LZ, R, seed=3, plant=plant)
    ref = np.fft.rfft(x, 2 * R * LZ)
    assert np.abs(X - ref).max() > 1e-3 * np.abs(ref).max()
