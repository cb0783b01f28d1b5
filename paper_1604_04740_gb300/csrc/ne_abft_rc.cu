// Row/column checksum ABFT of the products C_b = A_b B (the "ABFT RC-check"
// comparator the paper measures against in Sec. V, after Huang and Abraham):
// the checksum row e^T A_b and the checksum column B e (encoding), the border
// of the full-checksum matrix -- C_b e = A_b (B e), e^T C_b = (e^T A_b) B and
// the corner -- as matrix-vector products, one pass over C_b for its row and
// column sums, the consistency flags, and single-error correction.
//
// All sums are exact in wrapping 64-bit arithmetic: the true values fit the
// int64 words for the value ranges the comparator is used with, and a
// mismatch of the low 64 bits implies a mismatch of the exact values.
#include "ne_common.cuh"

namespace {

using namespace ne;

constexpr int kThreads = 256;
constexpr int kRows = 64;         // rows per block of the column sums of A
constexpr int kBand = 32;         // rows per block of the C pass

__device__ __forceinline__ void add64(int64_t* p, uint64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ac[b][t] += sum of rows [y*kRows, (y+1)*kRows) of column t of A_b
__global__ void __launch_bounds__(kThreads) k_rc_colsum_A(const int32_t* __restrict__ A, int64_t* ac, int64_t m,
                                                          int64_t k) {
    const int64_t b = blockIdx.z;
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= k) return;
    const int64_t i0 = (int64_t)blockIdx.y * kRows;
    const int64_t i1 = i0 + kRows < m ? i0 + kRows : m;
    const int32_t* Ab = A + b * m * k;
    uint64_t s = 0;
    for (int64_t i = i0; i < i1; i++) s += (uint64_t)(int64_t)__ldg(Ab + i * k + t);
    add64(ac + b * k + t, s);
}

// br[t] = sum_j B[t][j]: one warp per row
__global__ void __launch_bounds__(kThreads) k_rc_rowsum_B(const int8_t* __restrict__ B, int64_t* br, int64_t k,
                                                          int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (t >= k) return;
    const int lane = threadIdx.x & 31;
    uint64_t s = 0;
    for (int64_t j = lane; j < n; j += 32) s += (uint64_t)(int64_t)__ldg(B + t * n + j);
    s = warp_sum(s);
    if (lane == 0) br[t] = (int64_t)s;
}

// row_chk[b][i] = sum_t A_b[i][t] br[t]: one warp per row
__global__ void __launch_bounds__(kThreads) k_rc_row_checksums(const int32_t* __restrict__ A,
                                                               const int64_t* __restrict__ br, int64_t* work,
                                                               int64_t m, int64_t k, int64_t n) {
    const int64_t b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (i >= m) return;
    const int lane = threadIdx.x & 31;
    const int32_t* row = A + (b * m + i) * k;
    uint64_t s = 0;
    for (int64_t t = lane; t < k; t += 32) s += (uint64_t)(int64_t)__ldg(row + t) * (uint64_t)__ldg(br + t);
    s = warp_sum(s);
    if (lane == 0) work[b * 2 * (m + n + 1) + i] = (int64_t)s;
}

// col_chk[b][j] += sum over rows [y*kRows, ...) of ac[b][t] B[t][j]
__global__ void __launch_bounds__(kThreads) k_rc_col_checksums(const int8_t* __restrict__ B,
                                                               const int64_t* __restrict__ ac, int64_t* work,
                                                               int64_t m, int64_t k, int64_t n) {
    const int64_t b = blockIdx.z;
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j >= n) return;
    const int64_t t0 = (int64_t)blockIdx.y * kRows;
    const int64_t t1 = t0 + kRows < k ? t0 + kRows : k;
    uint64_t s = 0;
    for (int64_t t = t0; t < t1; t++) s += (uint64_t)__ldg(ac + b * k + t) * (uint64_t)(int64_t)__ldg(B + t * n + j);
    add64(work + b * 2 * (m + n + 1) + m + j, s);
}

// One block per product, after both checksum kernels: the corner
// sum_t ac[b][t] br[t], and the consistency of the border itself -- the sum
// of the column checksums and the sum of the row checksums against the
// corner -- kept as two bits in the last word of the product's work area
// (bit 0: the checksum row, bit 1: the checksum column).
__global__ void __launch_bounds__(kThreads) k_rc_corner(const int64_t* __restrict__ ac, const int64_t* __restrict__ br,
                                                        int64_t* work, int64_t m, int64_t k, int64_t n) {
    __shared__ uint64_t red[3][kThreads / 32];
    const int64_t b = blockIdx.x;
    int64_t* wb = work + b * 2 * (m + n + 1);
    uint64_t s = 0, sr = 0, sc = 0;
    for (int64_t t = threadIdx.x; t < k; t += kThreads) s += (uint64_t)ac[b * k + t] * (uint64_t)br[t];
    for (int64_t i = threadIdx.x; i < m; i += kThreads) sr += (uint64_t)wb[i];
    for (int64_t j = threadIdx.x; j < n; j += kThreads) sc += (uint64_t)wb[m + j];
    s = warp_sum(s);
    sr = warp_sum(sr);
    sc = warp_sum(sc);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s;
        red[1][threadIdx.x >> 5] = sr;
        red[2][threadIdx.x >> 5] = sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t v[3] = {0, 0, 0};
        for (int w = 0; w < kThreads / 32; w++)
            for (int q = 0; q < 3; q++) v[q] += red[q][w];
        wb[m + n] = (int64_t)v[0];
        wb[2 * (m + n + 1) - 1] = (int64_t)((v[2] != v[0] ? 1 : 0) | (v[1] != v[0] ? 2 : 0));
    }
}

// One pass over C_b: a block takes a band of kBand rows x 256 columns; every
// warp sums 4 of its rows (warp reduction, one atomic per row and block) and
// keeps 8 column partials per lane, combined across warps in shared memory
// (one atomic per column and block).
__global__ void __launch_bounds__(kThreads) k_rc_sums_C(const int64_t* __restrict__ C, int64_t* work, int64_t m,
                                                        int64_t n) {
    __shared__ uint64_t colp[kThreads / 32][kThreads];
    const int64_t b = blockIdx.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.x * kThreads;
    const int64_t i0 = (int64_t)blockIdx.y * kBand;
    const int64_t* Cb = C + b * m * n;
    int64_t* wb = work + b * 2 * (m + n + 1);
    uint64_t cs[8];
#pragma unroll
    for (int e = 0; e < 8; e++) cs[e] = 0;
    constexpr int rows_per_warp = kBand / (kThreads / 32);
#pragma unroll
    for (int rr = 0; rr < rows_per_warp; rr++) {
        const int64_t i = i0 + warp * rows_per_warp + rr;
        if (i >= m) break;
        uint64_t rs = 0;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int64_t j = j0 + e * 32 + lane;
            if (j < n) {
                const uint64_t v = (uint64_t)__ldcs(Cb + i * n + j);
                rs += v;
                cs[e] += v;
            }
        }
        rs = warp_sum(rs);
        if (lane == 0) add64(wb + (m + n + 1) + i, rs);
    }
#pragma unroll
    for (int e = 0; e < 8; e++) colp[warp][e * 32 + lane] = cs[e];
    __syncthreads();
    const int64_t j = j0 + threadIdx.x;
    if (j < n) {
        uint64_t v = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) v += colp[w][threadIdx.x];
        add64(wb + (m + n + 1) + m + j, v);
    }
}

// Consistency flags: row i < m compares its sum with row_chk[i], row m the
// sum of the column checksums with the corner; column j < n its sum with
// col_chk[j], column n the sum of the row checksums with the corner.
__global__ void __launch_bounds__(kThreads) k_rc_flags(const int64_t* __restrict__ work, uint32_t* row_bad,
                                                       uint32_t* col_bad, unsigned long long* nbad, int64_t m,
                                                       int64_t n) {
    const int64_t b = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t* wb = work + b * 2 * (m + n + 1);
    const int64_t* chk = wb;                  // row_chk [m], col_chk [n], corner
    const int64_t* sum = wb + (m + n + 1);    // row sums [m], column sums [n]
    const int64_t rw = (m + 1 + 31) / 32, cw = (n + 1 + 31) / 32;
    // rw*32 row slots (rows 0..m) followed by cw*32 column slots (columns 0..n):
    // a warp's 32 slots lie on one side and fill one bitmap word
    const int64_t slot = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    bool bad = false;
    if (slot < rw * 32) {
        const int64_t i = slot;
        if (i < m) bad = chk[i] != sum[i];
        else if (i == m) bad = (wb[2 * (m + n + 1) - 1] & 1) != 0;
        const uint32_t word = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) row_bad[b * rw + slot / 32] = word;
    } else if (slot < (rw + cw) * 32) {
        const int64_t j = slot - rw * 32;
        if (j < n) bad = chk[m + j] != sum[m + j];
        else if (j == n) bad = (wb[2 * (m + n + 1) - 1] & 2) != 0;
        const uint32_t word = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) col_bad[b * cw + j / 32] = word;
    }
    if (nbad) {
        const uint32_t word = __ballot_sync(0xffffffffu, bad);
        if (lane == 0 && word) atomicAdd(nbad + (slot < rw * 32 ? 0 : 1), (unsigned long long)__popc(word));
    }
}

// Single-error correction, one block per product: exactly one inconsistent
// row i and one inconsistent column j locate the faulty entry; for i < m and
// j < n it is C[i][j] and is corrected by row_chk[i] - rowsum[i] (the sums
// include the faulty value).  A fault located in the checksum border leaves C
// unchanged.
__global__ void __launch_bounds__(kThreads) k_rc_correct(int64_t* C, const int64_t* __restrict__ work,
                                                         const uint32_t* __restrict__ row_bad,
                                                         const uint32_t* __restrict__ col_bad,
                                                         unsigned long long* ncorrected, int64_t m, int64_t n) {
    __shared__ unsigned long long cnt[2], where[2];
    const int64_t b = blockIdx.x;
    const int64_t rw = (m + 1 + 31) / 32, cw = (n + 1 + 31) / 32;
    if (threadIdx.x < 2) {
        cnt[threadIdx.x] = 0;
        where[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    for (int64_t w = threadIdx.x; w < rw + cw; w += kThreads) {
        const int side = w < rw ? 0 : 1;
        const uint32_t word = side == 0 ? row_bad[b * rw + w] : col_bad[b * cw + (w - rw)];
        if (word) {
            atomicAdd(&cnt[side], (unsigned long long)__popc(word));
            const unsigned long long pos = (unsigned long long)((side == 0 ? w : w - rw) * 32 + (__ffs(word) - 1));
            atomicExch(&where[side], pos);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && cnt[0] == 1 && cnt[1] == 1) {
        const int64_t i = (int64_t)where[0], j = (int64_t)where[1];
        if (i < m && j < n) {
            const int64_t* wb = work + b * 2 * (m + n + 1);
            const uint64_t fix = (uint64_t)wb[i] - (uint64_t)wb[(m + n + 1) + i];
            int64_t* p = C + (b * m + i) * n + j;
            *p = (int64_t)((uint64_t)*p + fix);
            if (ncorrected) atomicAdd(ncorrected, 1ull);
        }
    }
}

ne_status rc_sizes(int64_t batch, int64_t m, int64_t k, int64_t n, const char* who) {
    if (batch < 0 || m < 0 || k < 0 || n < 0) return fail(NE_EINVAL, "%s: negative size", who);
    if (batch > 65535) return fail(NE_EINVAL, "%s: batch %lld exceeds 65535 products", who, (long long)batch);
    if ((m + kRows - 1) / kRows > 65535 || (k + kRows - 1) / kRows > 65535 || (m + kBand - 1) / kBand > 65535)
        return fail(NE_EINVAL, "%s: sizes exceed the launch grid", who);
    return NE_OK;
}

}  // namespace

extern "C" ne_status ne_abft_rc_encode(const int32_t* A, const int8_t* B, int64_t* ac, int64_t* br, int64_t batch,
                                       int64_t m, int64_t k, int64_t n, cudaStream_t s) {
    ne_status st = rc_sizes(batch, m, k, n, "ne_abft_rc_encode");
    if (st) return st;
    if (batch == 0 || k == 0) return NE_OK;
    if (!ac || !br || (m > 0 && !A) || (n > 0 && !B)) return fail(NE_EINVAL, "ne_abft_rc_encode: null pointer");
    if (cudaMemsetAsync(ac, 0, (size_t)batch * k * sizeof(int64_t), s) != cudaSuccess)
        return check_launch("ne_abft_rc_encode: zero");
    if (m > 0) {
        dim3 g((unsigned)((k + kThreads - 1) / kThreads), (unsigned)((m + kRows - 1) / kRows), (unsigned)batch);
        k_rc_colsum_A<<<g, kThreads, 0, s>>>(A, ac, m, k);
    }
    k_rc_rowsum_B<<<(unsigned)((k + 7) / 8), kThreads, 0, s>>>(B, br, k, n);
    return check_launch("ne_abft_rc_encode");
}

extern "C" ne_status ne_abft_rc_check(const int64_t* C, const int32_t* A, const int8_t* B, const int64_t* ac,
                                      const int64_t* br, int64_t* work, uint32_t* row_bad, uint32_t* col_bad,
                                      uint64_t* nbad, int64_t batch, int64_t m, int64_t k, int64_t n,
                                      cudaStream_t s) {
    ne_status st = rc_sizes(batch, m, k, n, "ne_abft_rc_check");
    if (st) return st;
    if (!work || !row_bad || !col_bad) return fail(NE_EINVAL, "ne_abft_rc_check: null pointer");
    unsigned long long* nb = reinterpret_cast<unsigned long long*>(nbad);
    if (nb && cudaMemsetAsync(nb, 0, 2 * sizeof(*nb), s) != cudaSuccess) return check_launch("ne_abft_rc_check: reset");
    if (batch == 0) return NE_OK;
    if ((m > 0 && k > 0 && !A) || (k > 0 && n > 0 && !B) || (m > 0 && n > 0 && !C) || (k > 0 && (!ac || !br)))
        return fail(NE_EINVAL, "ne_abft_rc_check: null pointer");
    if (cudaMemsetAsync(work, 0, (size_t)batch * 2 * (m + n + 1) * sizeof(int64_t), s) != cudaSuccess)
        return check_launch("ne_abft_rc_check: zero");
    if (m > 0 && k > 0) {
        dim3 g((unsigned)((m + 7) / 8), (unsigned)batch);
        k_rc_row_checksums<<<g, kThreads, 0, s>>>(A, br, work, m, k, n);
    }
    if (n > 0 && k > 0) {
        dim3 g((unsigned)((n + kThreads - 1) / kThreads), (unsigned)((k + kRows - 1) / kRows), (unsigned)batch);
        k_rc_col_checksums<<<g, kThreads, 0, s>>>(B, ac, work, m, k, n);
    }
    k_rc_corner<<<(unsigned)batch, kThreads, 0, s>>>(ac, br, work, m, k, n);
    if (m > 0 && n > 0) {
        dim3 g((unsigned)((n + kThreads - 1) / kThreads), (unsigned)((m + kBand - 1) / kBand), (unsigned)batch);
        k_rc_sums_C<<<g, kThreads, 0, s>>>(C, work, m, n);
    }
    const int64_t slots = ((m + 1 + 31) / 32 + (n + 1 + 31) / 32) * 32;
    dim3 g((unsigned)((slots + kThreads - 1) / kThreads), (unsigned)batch);
    k_rc_flags<<<g, kThreads, 0, s>>>(work, row_bad, col_bad, nb, m, n);
    return check_launch("ne_abft_rc_check");
}

extern "C" ne_status ne_abft_rc_correct(int64_t* C, const int64_t* work, const uint32_t* row_bad,
                                        const uint32_t* col_bad, uint64_t* ncorrected, int64_t batch, int64_t m,
                                        int64_t n, cudaStream_t s) {
    ne_status st = rc_sizes(batch, m, 0, n, "ne_abft_rc_correct");
    if (st) return st;
    unsigned long long* nc = reinterpret_cast<unsigned long long*>(ncorrected);
    if (nc && cudaMemsetAsync(nc, 0, sizeof(*nc), s) != cudaSuccess) return check_launch("ne_abft_rc_correct: reset");
    if (batch == 0) return NE_OK;
    if (!work || !row_bad || !col_bad || (m > 0 && n > 0 && !C)) return fail(NE_EINVAL, "ne_abft_rc_correct: null pointer");
    k_rc_correct<<<(unsigned)batch, kThreads, 0, s>>>(C, work, row_bad, col_bad, nc, m, n);
    return check_launch("ne_abft_rc_correct");
}
