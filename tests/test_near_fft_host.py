"""The algebra of the near zone by FFT (Sec. 3: the near zone of a regular
grid by an FFT with non-periodic boundaries on a doubled grid), on the host:
per pair of neighbour leaves, the 8^3 masses zero-padded to 16^3 and the
kernel placed at lag mod 16 give, summed over the 27 neighbours on the
spectra, exactly the direct near-zone sum; and for kernels that are even
(Phi) or odd (g) under lag -> -lag, the spectra of opposite offsets are
+-conjugates, the symmetry the spectral sums use to take the offsets in
pairs.  numpy only; no GPU."""
import numpy as np

S, M = 8, 16


def _kernels(seed):
    # four fields with the near table's parities: G even, -dG/dx_i odd in x_i
    # (zero at x_i = 0) and even in the other two components
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(2 * S, 2 * S, 2 * S, 4))
    a[:, :, 0, 1] = 0.0
    a[:, 0, :, 2] = 0.0
    a[0, :, :, 3] = 0.0

    def K(f, dx, dy, dz):
        t = a[np.abs(dz), np.abs(dy), np.abs(dx), f]
        sign = 1.0 if f == 0 else np.sign((dx, dy, dz)[f - 1])
        return sign * t
    return K


def _kernel_spectrum(K, f, o):
    lag = lambda v: v if v < S else v - M
    grid = np.zeros((M, M, M))
    for vz in range(M):
        for vy in range(M):
            for vx in range(M):
                if S in (vx, vy, vz):
                    continue
                grid[vz, vy, vx] = K(f, lag(vx) - S * o[0], lag(vy) - S * o[1], lag(vz) - S * o[2])
    return np.fft.fftn(grid)


def test_doubled_grid_convolution_is_the_direct_near_sum():
    nl = 3                                  # 3^3 leaves, periodic: every neighbour distinct
    K = _kernels(3)
    m = np.random.default_rng(4).normal(size=(nl * S,) * 3)
    offs = [(ox, oy, oz) for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)]
    f = 1                                   # an odd field (g_x) exercises the signs
    khat = {o: _kernel_spectrum(K, f, o) for o in offs}
    r = np.arange(S)
    for T in [(0, 0, 0), (2, 1, 0)]:        # target leaves (x, y, z)
        acc = np.zeros((M, M, M), complex)
        for o in offs:
            sx, sy, sz = [(T[i] + o[i]) % nl for i in range(3)]
            pad = np.zeros((M, M, M))
            pad[:S, :S, :S] = m[sz * S:(sz + 1) * S, sy * S:(sy + 1) * S, sx * S:(sx + 1) * S]
            acc += khat[o] * np.fft.fftn(pad)
        got = np.fft.ifftn(acc).real[:S, :S, :S]
        ref = np.zeros((S, S, S))
        for o in offs:
            sx, sy, sz = [(T[i] + o[i]) % nl for i in range(3)]
            src = m[sz * S:(sz + 1) * S, sy * S:(sy + 1) * S, sx * S:(sx + 1) * S]
            for tz in r:
                for ty in r:
                    for tx in r:
                        kk = K(f, tx - r[None, None, :] - S * o[0], ty - r[None, :, None] - S * o[1],
                               tz - r[:, None, None] - S * o[2])
                        ref[tz, ty, tx] += float((kk * src).sum())
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_opposite_offsets_have_conjugate_spectra():
    K = _kernels(5)
    for o in [(1, 0, 0), (1, -1, 1), (0, 1, -1)]:
        mo = tuple(-x for x in o)
        for f in range(4):
            s = 1.0 if f == 0 else -1.0
            a, b = _kernel_spectrum(K, f, mo), _kernel_spectrum(K, f, o)
            assert np.abs(a - s * np.conj(b)).max() <= 1e-12 * np.abs(b).max()
