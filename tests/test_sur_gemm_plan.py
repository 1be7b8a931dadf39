"""Host-side check of the surrogate training GEMM's data movement on the
tensor cores: the index arithmetic of its shared-memory fill (K-major and
MN-major sources, the in-register transpose of 8 x 8 blocks) is evaluated for
every thread of a CTA, and the stage images are read back through the
matrix descriptors the kernel gives its MMAs (start address, 128-byte
K-direction core-matrix offset, 1024-byte 8-row-group offset).  Every
global read stays inside its operand, every shared-memory write inside its
16 KB stage tile, every tile byte is written exactly once, and the product
decoded from the descriptors equals A B^T for all three operand layouts the
training pass uses.  Mirrors the arithmetic of gemm_tc_kernel and
load_stage in csrc/bte_sur_kernels.cu; the last test does the same for the
inference kernel's operand and weight layouts (csrc/bte_sur_tc.cu)."""
import numpy as np
import pytest

GM = GN = 128
GK = 64
THREADS = 256
CORE = 128
GROUP = (GK // 8) * CORE
TILE = GM * GK * 2


def gcanon(r, k):
    return ((r >> 3) * (GK // 8) + (k >> 3)) * CORE + (r & 7) * 16 + (k & 7) * 2


def fill_stage(src, ld, row0, k0, mn, first, extent_rows, extent_k):
    """Byte image (as bf16 element slots) of one stage tile written by the
    CTA's threads; src is the flat operand, element (row, k) at
    row * ld + k (K-major) or k * ld + row (MN-major)."""
    img = np.full(TILE // 2, -1, dtype=np.int64)
    writes = np.zeros(TILE // 2, dtype=np.int64)
    for t in range(THREADS):
        if not mn:
            for q in range(4):
                c = t + q * THREADS
                r, kc = (c & 7) + 8 * (c >> 6), (c >> 3) & 7
                g0 = (row0 + r) * ld + k0 + kc * 8
                assert 0 <= row0 + r < extent_rows and k0 + kc * 8 + 7 < extent_k
                assert g0 % 8 == 0  # 16-byte aligned vector load
                d = gcanon(r, kc * 8)
                assert d % 16 == 0 and 0 <= d and d + 16 <= TILE
                for e in range(8):
                    img[d // 2 + e] = src[g0 + e]
                    writes[d // 2 + e] += 1
        else:
            b = t - first
            if b < 0 or b >= 128:
                continue
            rb, kb = b & 15, b >> 4
            w = []
            for i in range(8):
                g0 = (k0 + kb * 8 + i) * ld + row0 + rb * 8
                assert k0 + kb * 8 + i < extent_k and row0 + rb * 8 + 7 < extent_rows
                assert g0 % 8 == 0
                w.append(src[g0:g0 + 8])
            dst = (rb * (GK // 8) + kb) * CORE
            for j in range(8):
                d = dst + j * 16
                assert d + 16 <= TILE
                # row j of the core matrix: element j of input rows 0..7
                for i in range(8):
                    img[d // 2 + i] = w[i][j]
                    writes[d // 2 + i] += 1
    assert np.all(writes == 1), "every element slot of the stage written exactly once"
    return img


def decode(img, rows):
    """Operand [rows][GK] as the MMAs read it: K-step ks starts at byte
    ks * 256, K-adjacent core matrices 128 bytes apart, 8-row groups 1024."""
    out = np.zeros((rows, GK), dtype=np.int64)
    for ks in range(GK // 16):
        start = ks * 2 * CORE
        for r in range(rows):
            for kk in range(16):
                byte = start + (kk >> 3) * CORE + (r >> 3) * GROUP + (r & 7) * 16 + (kk & 7) * 2
                out[r, ks * 16 + kk] = img[byte // 2]
    return out


@pytest.mark.parametrize("amn,bmn", [(False, False), (False, True), (True, True)])
def test_stage_fill_and_descriptors_give_a_times_b_transposed(amn, bmn):
    rng = np.random.default_rng(7)
    M, N, K = 256, 256, 128
    A = rng.integers(-50, 50, size=(M, K))   # logical A[m][k]
    B = rng.integers(-50, 50, size=(N, K))   # logical B[n][k]
    a_src = (A.T if amn else A).ravel()       # stored [k][m] or [m][k]
    b_src = (B.T if bmn else B).ravel()
    lda = M if amn else K
    ldb = N if bmn else K
    C = np.zeros((M, N), dtype=np.int64)
    for by in range(M // GM):
        for bx in range(N // GN):
            m0, n0 = by * GM, bx * GN
            acc = np.zeros((GM, GN), dtype=np.int64)
            for kt in range(K // GK):
                ia = fill_stage(a_src, lda, m0, kt * GK, amn, 0, M, K)
                ib = fill_stage(b_src, ldb, n0, kt * GK, bmn, 128 if amn else 0, N, K)
                acc += decode(ia, GM) @ decode(ib, GN).T
            C[m0:m0 + GM, n0:n0 + GN] = acc
    assert np.array_equal(C, A @ B.T)


def test_inference_weights_and_operand_decode_through_descriptors():
    """Inference kernel (csrc/bte_sur_tc.cu): W2/W3 stored as two halves of
    128 output rows ([128][256] each) and h stored [128 rows][256], both
    canonical with 8-row groups 4096 bytes apart.  Decoding the MMAs of
    K-step ks (start = base + ks * 256; K-adjacent core matrices 128 bytes
    apart) for weight half hh gives back h[r][16 ks + kk] and
    W[128 hh + n][16 ks + kk], so the 2 x 16 MMAs of a layer compute h W^T."""
    def canon(r, k):
        return ((r >> 3) * 32 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2

    rng = np.random.default_rng(3)
    W = rng.integers(-1000, 1000, size=(256, 256))
    h = rng.integers(-1000, 1000, size=(128, 256))
    halves = []
    for hh in range(2):
        img = np.full(128 * 256, -10**9, dtype=np.int64)
        for n in range(128):
            for k in range(256):
                off = canon(n, k)
                assert 0 <= off < 65536 and off % 2 == 0
                img[off // 2] = W[128 * hh + n, k]
        assert np.all(img >= -1000), "every byte of the half written"
        halves.append(img)
    himg = np.full(128 * 256, -10**9, dtype=np.int64)
    for r in range(128):
        for k in range(256):
            himg[canon(r, k) // 2] = h[r, k]
    assert np.all(himg >= -1000), "every byte of h written"

    def read(img, ks, r, kk):
        return img[(ks * 256 + (kk >> 3) * 128 + (r >> 3) * 4096 + (r & 7) * 16 + (kk & 7) * 2) // 2]

    acc = np.zeros((128, 256), dtype=np.int64)
    for hh in range(2):
        for ks in range(16):
            a = np.array([[read(himg, ks, r, kk) for kk in range(16)] for r in range(128)])
            b = np.array([[read(halves[hh], ks, n, kk) for kk in range(16)] for n in range(128)])
            acc[:, 128 * hh:128 * hh + 128] += a @ b.T
    assert np.array_equal(acc, h @ W.T)
