// Ragged batches of independent jobs (products and circular convolutions of
// entangled streams, each with its own M, l and sizes) in one persistent
// launch.  Sec. IV of the paper processes long streams and large products as
// many independent blocks; every block is entangled, operated on (Eq. 10),
// extracted and checked (Eq. 17-20, Eq. 24) on its own, so a batch is a
// list of such blocks of different shapes.
//
//   ne_batch_plan (host): per job l (Eq. 13/14 from the job's bound) and the
//     digit plan; digit-plane arena layout; entangle segments; operation
//     tiles (ordered by cost when asked); tables copied to the workspace.
//   ne_batch_run (device, graph-capturable): clear the tile counters and the
//     flag bitmaps; one launch entangles every segment into digit planes;
//     two persistent launches, one over the product tiles (16 x 64 outputs,
//     all M*S planes; 3 CTAs per SM) and one over the convolution tiles (up
//     to 1024 outputs, all planes, ne_cconv_tile.cuh): each CTA takes the
//     next tile of its list from an atomic counter and runs it with the fused
//     extract/check or fused recovery of its job.
//   Long convolutions (N >= the plan's ntt_min_n) skip the tiles and run as
//     exact two-prime transforms (ne_ntt_any.cu) in the launches that follow,
//     with the same epilogues and the same fault hook.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ne_cconv_tile.cuh"
#include "ne_entangle.cuh"
#include "ne_extract.cuh"
#include "ne_mma.cuh"
#include "ne_ntt_any.cuh"

namespace {

using namespace ne;

constexpr int THREADS = 256;
constexpr int SEG = 8192;        // positions per entangle segment
constexpr int MS_MAX = 10;       // M <= 5 streams x S <= 2 digits

struct DevJob {
    int32_t kind, M, l, S, MS, rows, cols, k, N, r, fuse;
    int32_t kc;                  // products: the inputs' k; k itself is the digit planes' and
                                 // G^T's row length, kc rounded up to 16 (zero padded)
    int32_t shift[NE_MAX_DIGITS];
    FastPlan fp;
    int64_t c_off, op_off, out_off, flag_off, plane_off, npos, nout, fault_begin, fault_end;
    int64_t gt_off;              // products: G transposed, [cols][k], in the planes arena
};

struct DevTile {
    int32_t job, kind, a, b;     // product: row tile, column tile; convolution: output chunk, blocks
};

constexpr int SEG_ENTANGLE = 0, SEG_TRANSPOSE = 1;
constexpr int SEG_ROWS = 2;      // a product whose k is not a multiple of 16: whole rows, padded
constexpr int TT = 64;           // G transpose tiles: TT k x TT columns
constexpr int TT_PER_SEG = 16;
constexpr int TT_ROUND = 4;      // transpose tiles loaded together

struct DevSeg {
    int32_t job, kind;
    int64_t start, count;        // entangle: positions of every stream of the job; transpose: tiles;
                                 // rows: rows of every stream
};

struct Layout {
    int64_t jobs, tiles, segs, planes, ntt_table, ntt_ws, total;
};

int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

Layout layout(int64_t njobs, int64_t ntiles, int64_t nsegs, int64_t plane_bytes, int64_t nntt = 0,
              int64_t ntt_ws_bytes = 0) {
    Layout L;
    L.jobs = 256;
    L.tiles = align256(L.jobs + njobs * (int64_t)sizeof(DevJob));
    L.segs = align256(L.tiles + ntiles * (int64_t)sizeof(DevTile));
    L.planes = align256(L.segs + nsegs * (int64_t)sizeof(DevSeg));
    L.ntt_table = align256(L.planes + plane_bytes);
    L.ntt_ws = align256(L.ntt_table + nntt * (int64_t)sizeof(NJob));
    L.total = align256(L.ntt_ws + ntt_ws_bytes);
    return L;
}

// ---- the product tile: 16 x 64 outputs of every digit plane, 8 warps -------------------
//
// mma.sync wants both operands k-major; the entangle launch writes each
// product job's G transposed ([cols][k]) next to its digit planes, so both
// operand tiles of a k step arrive by cp.async as 128-byte k-rows, unpadded in
// shared memory, the 16-byte chunk c of row r at chunk c ^ sw(r).  sw takes 8
// distinct values on every aligned group of 8 rows (the rows of one ldmatrix
// phase), so the fragment loads have no bank conflicts.

namespace bgemm {

constexpr int BM = 16, BN = 64, BK = 128, STAGES = 2, RB = 128, SB = 72;
constexpr int CTAS = 3;            // resident CTAs per SM of the product launch
constexpr int FCAP = 64;           // faults of one tile kept in shared memory
constexpr int UPW = 3;            // (plane, column half) units per warp: 2 * MS_MAX / 8, rounded up

// the pipeline, or after the main loop the stash and the tile's fault list
__host__ __device__ constexpr int smem_bytes(int MS) {
    return (STAGES * (MS * BM * RB + BN * RB)) > (MS * BM * SB * 4 + 4 * FCAP + 32)
               ? (STAGES * (MS * BM * RB + BN * RB))
               : (MS * BM * SB * 4 + 4 * FCAP + 32);
}

__device__ __forceinline__ int sw(int r) { return ((r >> 2) ^ r) & 7; }


struct TileArgs {
    const int8_t* planes;        // [M][S][rows][k]
    const int8_t* GT;            // G transposed: [cols][k]
    int64_t* out;                // [M][rows][cols]
    uint32_t* flags;             // bitmap over i * cols + j (pre-zeroed) or null
    unsigned long long* nflag;
    const int64_t* fault_pos;    // sorted positions i * cols + j, or null
    const int32_t* fault_stream;
    const int32_t* fault_bit;
    int64_t nfault;
    int rows, cols, k, M, S, MS, l, r, fuse;
    int shift[NE_MAX_DIGITS];
};

// first index in [0, n) with pos[index] >= key (pos sorted ascending), by the
// 32 lanes of a warp together: each round probes 32 points of the interval
// left and keeps the part between the last probe below key and the first at
// or above it
__device__ __forceinline__ int64_t warp_lower_bound(const int64_t* pos, int64_t n, int64_t key) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t len = hi - lo;
        const int64_t p = lo + len * (lane + 1) / 33;           // nondecreasing in lane, in [lo, hi)
        const unsigned below = __ballot_sync(0xffffffffu, pos[p] < key);
        const int c = __popc(below);                             // a prefix of the lanes
        const int64_t p_last = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0);
        const int64_t p_next = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
        if (c > 0) lo = p_last + 1;
        if (c < 32) hi = p_next;
    }
    return lo;
}

// The faults of a tile: the first warp locates the job's faults in the
// tile's row band, keeps those inside its columns as (local index, stream,
// bit) and returns their count, or -1 when there are more than FCAP (then
// every position scans the band).
__device__ __forceinline__ int tile_faults(const TileArgs& a, int row0, int col0, int32_t* list, int* count,
                                           int64_t* band) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int64_t f0 = warp_lower_bound(a.fault_pos, a.nfault, (int64_t)row0 * a.cols + col0);
        const int64_t f1 = warp_lower_bound(a.fault_pos, a.nfault, (int64_t)(row0 + BM - 1) * a.cols + col0 + BN);
        int n = 0;
        for (int64_t f = f0 + lane; f - lane < f1; f += 32) {
            bool keep = false;
            int32_t e = 0;
            if (f < f1) {
                const int64_t pos = a.fault_pos[f];
                const int i = (int)(pos / a.cols), j = (int)(pos - (int64_t)i * a.cols);
                keep = j >= col0 && j < col0 + BN;
                e = (((i - row0) * BN + (j - col0)) << 16) | (a.fault_stream[f] << 8) | a.fault_bit[f];
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int at = n + __popc(m & ((1u << lane) - 1));
            if (keep && at < FCAP) list[at] = e;
            n += __popc(m);
        }
        if (lane == 0) {
            *count = n <= FCAP ? n : -1;
            band[0] = f0;
            band[1] = f1;
        }
    }
    __syncthreads();
    return *count;
}

// LT: the job's l when it is 8 or 16 (then every shift below is a constant;
// with two digits at shifts 0 and l, as the byte-aligned plans of int8-valued
// streams have, the recombination is one shift-add), else 0
template <int MT, int LT>
__device__ __forceinline__ void epilogue(const TileArgs& a, const int32_t* stash, int row0, int col0, uint8_t* spare) {
    const int M = MT ? MT : a.M;
    const int l = LT ? LT : a.l;
    const bool two = LT && a.S == 2 && a.shift[0] == 0 && a.shift[1] == LT;
    const int S = a.S;
    const int lane = threadIdx.x & 31;
    const bool check = (a.fuse == NE_FUSE_EXTRACT_CHECK);
    const bool need_r = (a.fuse != NE_FUSE_RECOVER);
    const int64_t plane = (int64_t)a.rows * a.cols;
    int32_t* flist = reinterpret_cast<int32_t*>(spare);
    int64_t* band = reinterpret_cast<int64_t*>(spare + 4 * FCAP);
    int* fcount = reinterpret_cast<int*>(spare + 4 * FCAP + 16);
    const int nf = a.nfault > 0 ? tile_faults(a, row0, col0, flist, fcount, band) : 0;
    for (int base = threadIdx.x & ~31; base < BM * BN; base += THREADS) {
        const int idx = base + lane;
        const int i = idx / BN, j = idx % BN;
        const int gi = row0 + i, gj = col0 + j;
        if (gi >= a.rows || gj >= a.cols) continue;
        const int32_t* sp = stash + i * SB + j;
        const int64_t pos = (int64_t)gi * a.cols + gj;
        int64_t rot[MT ? MT : 32], res[MT ? MT : 32];
#pragma unroll
        for (int jj = 0; jj < (MT ? MT : 32); jj++) {
            if (!MT && jj >= M) break;
            int m = a.r + jj;
            if (m >= M) m -= M;
            int64_t v = 0;
            if (jj > 0 || need_r) {
                if (two) {
                    v = (int64_t)sp[2 * m * BM * SB] + (int64_t)((uint64_t)(int64_t)sp[(2 * m + 1) * BM * SB] << LT);
                } else {
#pragma unroll
                    for (int s = 0; s < NE_MAX_DIGITS; s++)
                        if (s < S) v += cconv::shl64(sp[(m * S + s) * BM * SB], a.shift[s]);
                }
                if (nf > 0) {
                    for (int f = 0; f < nf; f++) {
                        const int32_t e = flist[f];
                        if ((e >> 16) == idx && ((e >> 8) & 0xff) == m) v ^= (int64_t)(1ull << (e & 0xff));
                    }
                } else if (nf < 0) {
                    for (int64_t f = band[0]; f < band[1]; f++)
                        if (a.fault_pos[f] == pos && a.fault_stream[f] == m) v ^= (int64_t)(1ull << a.fault_bit[f]);
                }
            }
            rot[jj] = v;
        }
        bool flag = false;
        if (a.fuse == NE_FUSE_NONE) {
            // the operation's words themselves (entangled delta, or the plain d)
#pragma unroll
            for (int jj = 0; jj < (MT ? MT : 32); jj++) {
                if (!MT && jj >= M) break;
                int m = a.r + jj;
                if (m >= M) m -= M;
                a.out[m * plane + pos] = rot[jj];
            }
            continue;
        }
        flag = extract_rot<MT>(rot, M, l, check, res);
#pragma unroll
        for (int jj = 0; jj < (MT ? MT : 32); jj++) {
            if (!MT && jj >= M) break;
            int m = a.r + jj;
            if (m >= M) m -= M;
            a.out[m * plane + pos] = res[jj];
        }
        if (flag) {
            if (a.flags) atomicOr(&a.flags[pos >> 5], 1u << (pos & 31));
            if (a.nflag) atomicAdd(a.nflag, 1ull);
        }
    }
}

template <int MT>
__device__ __forceinline__ void tile(const TileArgs& a, uint8_t* smem, int row0, int col0) {
    const int MS = a.MS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.k, rows = a.rows, cols = a.cols;
    const int KT = (K + BK - 1) / BK;
    const bool recover = (a.fuse == NE_FUSE_RECOVER);

    uint8_t* As = smem;                                    // [STAGES][MS][BM][RB]
    uint8_t* Bs = smem + STAGES * MS * BM * RB;            // [STAGES][BN][RB] (G transposed)
    const uint32_t As_s = smem_u32(As), Bs_s = smem_u32(Bs);

    // one k step of both operands: the digit-plane rows and the G^T rows
    // (columns col0 .. col0 + 63), 16-byte chunks, zero-filled outside
    auto load_AB = [&](int stage, int kt) {
        const int k0 = kt * BK;
        for (int e = tid; e < MS * BM * 8; e += THREADS) {
            const int c16 = e & 7, r = (e >> 3) % BM, pl = (e >> 3) / BM;
            const int gi = row0 + r, gk = k0 + 16 * c16;
            const bool ok = gi < rows && gk < K && !(recover && pl / a.S == a.r);
            const int8_t* src = a.planes + ((int64_t)pl * rows + (ok ? gi : 0)) * K + (ok ? gk : 0);
            cp_async16(As_s + ((stage * MS + pl) * BM + r) * RB + 16 * (c16 ^ sw(r)), src, ok ? 16 : 0);
        }
        for (int e = tid; e < BN * 8; e += THREADS) {
            const int c16 = e & 7, n = e >> 3;
            const int gn = col0 + n, gk = k0 + 16 * c16;
            const bool ok = gn < cols && gk < K;
            const int8_t* src = a.GT + (int64_t)(ok ? gn : 0) * K + (ok ? gk : 0);
            cp_async16(Bs_s + (stage * BN + n) * RB + 16 * (c16 ^ sw(n)), src, ok ? 16 : 0);
        }
    };
    int acc[UPW][4][4];
#pragma unroll
    for (int i = 0; i < UPW; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0;

#pragma unroll
    for (int st = 0; st < STAGES - 1; st++) {
        if (st < KT) load_AB(st, st);
        cp_async_commit();
    }
    // lane offsets of the fragment loads: A rows lane & 15 at chunk 2 ks + (lane >> 4);
    // G rows n(nj) at chunk 2 ks + ((lane >> 3) & 1)
    const int ar = lane & 15, ac = lane >> 4, bc = (lane >> 3) & 1;
    for (int kt = 0; kt < KT; kt++) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int pf = kt + STAGES - 1;
        if (pf < KT) load_AB(pf % STAGES, pf);
        cp_async_commit();
        const int st = kt % STAGES;
#pragma unroll
        for (int ks = 0; ks < BK / 32; ks++) {
            if (kt * BK + 32 * ks >= K) break;      // k is a multiple of 16: the rest of the tile is padding
            // every unit of a warp has the same column half (units w, w + 8, ...):
            // its G fragments are loaded once and used by each of its planes
            uint32_t bf[2][4];
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                const int n = 32 * (warp & 1) + 8 * (nj + (lane >> 4)) + (lane & 7);
                ldsm_x4(bf[nj >> 1], Bs_s + (st * BN + n) * RB + 16 * ((2 * ks + bc) ^ sw(n)));
            }
#pragma unroll
            for (int i = 0; i < UPW; i++) {
                const int u = warp + 8 * i;
                if (u >= 2 * MS) break;
                const int pl = u >> 1;
                if (recover && pl / a.S == a.r) continue;
                uint32_t af[4];
                ldsm_x4(af, As_s + ((st * MS + pl) * BM + ar) * RB + 16 * ((2 * ks + ac) ^ sw(ar)));
#pragma unroll
                for (int nj = 0; nj < 4; nj += 2) {
                    mma_s8(acc[i][nj], af, bf[nj >> 1][0], bf[nj >> 1][1]);
                    mma_s8(acc[i][nj + 1], af, bf[nj >> 1][2], bf[nj >> 1][3]);
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    int32_t* stash = reinterpret_cast<int32_t*>(smem);    // [MS][BM][SB]
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < UPW; i++) {
        const int u = warp + 8 * i;
        if (u >= 2 * MS) break;
        const int pl = u >> 1, nh = u & 1;
#pragma unroll
        for (int nj = 0; nj < 4; nj++)
#pragma unroll
            for (int h = 0; h < 4; h += 2)
                *reinterpret_cast<int2*>(stash + (pl * BM + gq + 8 * (h >> 1)) * SB + 32 * nh + 8 * nj + 2 * tq) =
                    make_int2(acc[i][nj][h], acc[i][nj][h + 1]);
    }
    __syncthreads();
    uint8_t* spare = smem + MS * BM * SB * 4;
    if (a.l == 16) epilogue<MT, 16>(a, stash, row0, col0, spare);
    else if (a.l == 8) epilogue<MT, 8>(a, stash, row0, col0, spare);
    else epilogue<MT, 0>(a, stash, row0, col0, spare);
}

}  // namespace bgemm

// ---- kernels -------------------------------------------------------------------------------

struct BatchK {
    const DevJob* jobs;
    const DevTile* tiles;
    const DevSeg* segs;
    int32_t* counter;            // [0]: product tiles taken, [1]: convolution tiles taken
    int8_t* planes;
    int ngemm, ntiles, nsegs;    // tiles [0, ngemm) are products, [ngemm, ntiles) convolutions
    const int32_t* c;
    const int8_t* ops;
    int64_t* out;
    uint32_t* flags;
    unsigned long long* nflag;
    const int64_t* fault_pos;
    const int32_t* fault_stream;
    const int32_t* fault_bit;
    int32_t* status;
};

template <int MT>
__device__ __forceinline__ bool entangle_segment(const BatchK& k, const DevJob* J, const DevSeg& sg) {
    const int64_t n = J->npos;
    const int32_t* cb = k.c + J->c_off;
    int8_t* pb = k.planes + J->plane_off;
    const FastPlan F = J->fp;
    const int l = J->l;
    uint32_t worst = 0;
    const int64_t q1 = (sg.start + sg.count) / 8;
    if (F.pmask == 0) {   // a plain job: digits of the raw streams
        for (int64_t q = sg.start / 8 + threadIdx.x; q < q1; q += THREADS)
            worst = max(worst, entangle_chunk8<MT, true>(cb + q * 8, pb + q * 8, n, l, F));
    } else {
        for (int64_t q = sg.start / 8 + threadIdx.x; q < q1; q += THREADS)
            worst = max(worst, entangle_chunk8<MT>(cb + q * 8, pb + q * 8, n, l, F));
    }
    return worst <= (uint32_t)F.hi - (uint32_t)F.lo;
}

// Rows [start, start + count) of a product job whose k is not a multiple of
// 16: the digit planes keep rows of k = kc rounded up to 16 so that the tiles
// stream them in 16-byte pieces; positions kc .. k - 1 hold the word 0 (every
// digit 0), which adds nothing to the products.  Inputs are read element by
// element (a row of kc int32 values need not start 16-byte aligned); each
// thread forms 8 positions of one row of every stream and stores 8 bytes per
// digit plane.
template <int MT>
__device__ __forceinline__ bool entangle_rows(const BatchK& k, const DevJob* J, const DevSeg& sg) {
    const int kc = J->kc, kp = J->k;
    const int64_t nin = (int64_t)J->rows * kc, npl = (int64_t)J->rows * kp;
    const int32_t* cb = k.c + J->c_off;
    int8_t* pb = k.planes + J->plane_off;
    const FastPlan F = J->fp;
    const int l = J->l;
    const bool plain = F.pmask == 0;
    uint32_t worst = 0;
    const int cpr = kp / 8;
    const int64_t nch = sg.count * cpr;
    for (int64_t q = threadIdx.x; q < nch; q += THREADS) {
        const int64_t row = sg.start + q / cpr;
        const int t0 = (int)(q % cpr) * 8;
        uint32_t v[MT][8];
#pragma unroll
        for (int m = 0; m < MT; m++)
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int t = t0 + e;
                v[m][e] = 0;
                if (t < kc) {
                    v[m][e] = (uint32_t)__ldg(cb + m * nin + row * kc + t);
                    worst = max(worst, v[m][e] - (uint32_t)F.lo);
                }
            }
#pragma unroll
        for (int m = 0; m < MT; m++) {
            const int pm = (m + MT - 1) % MT;
            uint32_t y[8];
#pragma unroll
            for (int e = 0; e < 8; e++) y[e] = v[m][e] + (plain ? 0u : v[pm][e] << l) + F.off;
#pragma unroll
            for (int s = 0; s < 4; s++) {
                if (s >= F.S) break;
                const uint32_t t = (uint32_t)F.byte_of[s];
                const uint32_t sel = t | ((t + 4) << 4);
                const uint32_t w0 = __byte_perm(__byte_perm(y[0], y[1], sel), __byte_perm(y[2], y[3], sel), 0x5410);
                const uint32_t w1 = __byte_perm(__byte_perm(y[4], y[5], sel), __byte_perm(y[6], y[7], sel), 0x5410);
                *reinterpret_cast<uint2*>(pb + (m * F.S + s) * npl + row * kp + t0) =
                    make_uint2(w0 ^ 0x80808080u, w1 ^ 0x80808080u);
            }
        }
    }
    return worst <= (uint32_t)F.hi - (uint32_t)F.lo;
}

// tiles [start, start + count) of G^T = the transpose of a product job's G
// ([k][cols] -> [cols][k], so the product tiles stream both operands k-major),
// TT_ROUND tiles per round so that each thread has 4 TT_ROUND loads in flight
__device__ __forceinline__ void transpose_segment(const BatchK& k, const DevJob* J, const DevSeg& sg,
                                                  uint8_t (*tile)[TT][TT + 4]) {
    const int K = J->kc, KP = J->k, cols = J->cols;
    const bool words = (cols & 3) == 0;        // rows of G start 4-byte aligned
    const int nct = (cols + TT - 1) / TT;
    const uint8_t* G = reinterpret_cast<const uint8_t*>(k.ops + J->op_off);
    uint8_t* GT = reinterpret_cast<uint8_t*>(k.planes + J->gt_off);
    for (int64_t t0 = sg.start; t0 < sg.start + sg.count; t0 += TT_ROUND) {
        const int nt = (int)min((int64_t)TT_ROUND, sg.start + sg.count - t0);
        // rows k0 .. k0 + 63 of G, 4 bytes per thread and step (rows are 4-byte aligned)
        uint32_t w[TT_ROUND][TT * TT / 4 / THREADS];
#pragma unroll
        for (int h = 0; h < TT_ROUND; h++) {
            const int64_t t = t0 + h;
            const int k0 = (int)(t / nct) * TT, c0 = (int)(t % nct) * TT;
#pragma unroll
            for (int i = 0; i < TT * TT / 4 / THREADS; i++) {
                const int e = threadIdx.x + i * THREADS;
                const int kr = e / (TT / 4), cw = e % (TT / 4);
                const int gk = k0 + kr, gc = c0 + 4 * cw;
                uint32_t x = 0;
                if (h < nt && gk < K && gc < cols) {
                    if (words) {
                        x = __ldg(reinterpret_cast<const uint32_t*>(G + (int64_t)gk * cols + gc));
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (gc + q < cols) x |= (uint32_t)__ldg(G + (int64_t)gk * cols + gc + q) << (8 * q);
                    }
                }
                w[h][i] = x;
            }
        }
#pragma unroll
        for (int h = 0; h < TT_ROUND; h++)
#pragma unroll
            for (int i = 0; i < TT * TT / 4 / THREADS; i++) {
                const int e = threadIdx.x + i * THREADS;
                *reinterpret_cast<uint32_t*>(&tile[h][e / (TT / 4)][4 * (e % (TT / 4))]) = w[h][i];
            }
        __syncthreads();
        // rows c0 .. c0 + 63 of G^T, 16 bytes (16 k) per thread and step; rows of KP
        // (a multiple of 16) bytes, the padding kc .. KP - 1 zero
        for (int h = 0; h < nt; h++) {
            const int64_t t = t0 + h;
            const int k0 = (int)(t / nct) * TT, c0 = (int)(t % nct) * TT;
            for (int e = threadIdx.x; e < TT * TT / 16; e += THREADS) {
                const int n = e / (TT / 16), kc = e % (TT / 16);
                const int gc = c0 + n, gk = k0 + 16 * kc;
                if (gc < cols && gk < KP) {
                    uint32_t o[4];
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        o[q] = (uint32_t)tile[h][16 * kc + 4 * q][n] | ((uint32_t)tile[h][16 * kc + 4 * q + 1][n] << 8) |
                               ((uint32_t)tile[h][16 * kc + 4 * q + 2][n] << 16) |
                               ((uint32_t)tile[h][16 * kc + 4 * q + 3][n] << 24);
                    *reinterpret_cast<uint4*>(GT + (int64_t)gc * KP + gk) = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(THREADS) k_batch_entangle(BatchK k) {
    __shared__ uint8_t tile[TT_ROUND][TT][TT + 4];
    bool ok = true;
    for (int si = blockIdx.x; si < k.nsegs; si += gridDim.x) {
        const DevSeg sg = k.segs[si];
        const DevJob* J = k.jobs + sg.job;
        if (sg.kind == SEG_TRANSPOSE) {
            transpose_segment(k, J, sg, tile);
            continue;
        }
        if (sg.kind == SEG_ROWS) {
            switch (J->M) {
                case 3: ok &= entangle_rows<3>(k, J, sg); break;
                case 4: ok &= entangle_rows<4>(k, J, sg); break;
                default: ok &= entangle_rows<5>(k, J, sg); break;
            }
            continue;
        }
        switch (J->M) {
            case 3: ok &= entangle_segment<3>(k, J, sg); break;
            case 4: ok &= entangle_segment<4>(k, J, sg); break;
            default: ok &= entangle_segment<5>(k, J, sg); break;
        }
    }
    if (!ok && k.status) atomicExch(k.status, (int32_t)NE_ERANGE);
}

__device__ __forceinline__ void fill_common(const BatchK& k, const DevJob* J, int64_t*& fpos, const int32_t*& fstr,
                                            const int32_t*& fbit, int64_t& nf) {
    if (k.fault_pos && J->fault_end > J->fault_begin) {
        fpos = const_cast<int64_t*>(k.fault_pos) + J->fault_begin;
        fstr = k.fault_stream + J->fault_begin;
        fbit = k.fault_bit + J->fault_begin;
        nf = J->fault_end - J->fault_begin;
    } else {
        fpos = nullptr;
        fstr = nullptr;
        fbit = nullptr;
        nf = 0;
    }
}

__device__ __forceinline__ void run_cconv(const BatchK& k, const DevJob* J, const DevTile& tl, uint8_t* smem) {
    cconv::TileArgs t;
    t.planes = k.planes + J->plane_off;
    t.g = k.ops + J->op_off;
    t.out = k.out + J->out_off;
    t.flags = (J->fuse == NE_FUSE_EXTRACT_CHECK && k.flags) ? k.flags + J->flag_off : nullptr;
    t.nflag = (J->fuse == NE_FUSE_EXTRACT_CHECK) ? k.nflag : nullptr;
    int64_t* fp;
    fill_common(k, J, fp, t.fault_stream, t.fault_bit, t.nfault);
    t.fault_pos = fp;
    t.fault_base = 0;
    t.N = J->N;
    t.M = J->M;
    t.S = J->S;
    t.MS = J->MS;
    t.l = J->l;
    t.r = J->r;
    t.fuse = J->fuse;
    t.flags_atomic = 1;
    t.craw = nullptr;     // the batch's digit planes come from its segment entangle
    t.status = nullptr;
#pragma unroll
    for (int i = 0; i < NE_MAX_DIGITS; i++) t.shift[i] = J->shift[i];
    const int NB = J->N / cconv::T;
    const int p0 = tl.a * tl.b;
    const int npb = min(tl.b, NB - p0);
    switch (J->M) {
        case 3: cconv::tile<10, 3>(t, smem, p0, npb); break;
        case 4: cconv::tile<10, 4>(t, smem, p0, npb); break;
        default: cconv::tile<10, 5>(t, smem, p0, npb); break;
    }
}

__device__ __forceinline__ void run_gemm(const BatchK& k, const DevJob* J, const DevTile& tl, uint8_t* smem) {
    bgemm::TileArgs t;
    t.planes = k.planes + J->plane_off;
    t.GT = k.planes + J->gt_off;
    t.out = k.out + J->out_off;
    t.flags = (J->fuse == NE_FUSE_EXTRACT_CHECK && k.flags) ? k.flags + J->flag_off : nullptr;
    t.nflag = (J->fuse == NE_FUSE_EXTRACT_CHECK) ? k.nflag : nullptr;
    int64_t* fp;
    fill_common(k, J, fp, t.fault_stream, t.fault_bit, t.nfault);
    t.fault_pos = fp;
    t.rows = J->rows;
    t.cols = J->cols;
    t.k = J->k;
    t.M = J->M;
    t.S = J->S;
    t.MS = J->MS;
    t.l = J->l;
    t.r = J->r;
    t.fuse = J->fuse;
#pragma unroll
    for (int i = 0; i < NE_MAX_DIGITS; i++) t.shift[i] = J->shift[i];
    switch (J->M) {
        case 3: bgemm::tile<3>(t, smem, tl.a * bgemm::BM, tl.b * bgemm::BN); break;
        case 4: bgemm::tile<4>(t, smem, tl.a * bgemm::BM, tl.b * bgemm::BN); break;
        default: bgemm::tile<5>(t, smem, tl.a * bgemm::BM, tl.b * bgemm::BN); break;
    }
}

// the product tiles, 3 CTAs per SM: while one CTA fills its pipeline or runs
// its epilogue, the others keep the tensor pipe busy
__global__ void __launch_bounds__(THREADS, bgemm::CTAS) k_batch_gemm(BatchK k) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(k.counter, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= k.ngemm) break;
        const DevTile tl = k.tiles[t];
        run_gemm(k, k.jobs + tl.job, tl, smem);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(THREADS, 2) k_batch_cconv(BatchK k) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = k.ngemm + atomicAdd(k.counter + 1, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= k.ntiles) break;
        const DevTile tl = k.tiles[t];
        run_cconv(k, k.jobs + tl.job, tl, smem);
        __syncthreads();
    }
}

// Balanced base-256 digits that occur among the values [lo, hi] themselves.
ne_status plain_digits(int32_t lo, int32_t hi, ne_digits* dg) {
    uint32_t used = 0;
    if ((int64_t)hi - lo <= 65536) {
        for (int64_t a = lo; a <= hi; a++) {
            int64_t x = a;
            for (int t = 0; t < 8 && x != 0; t++) {
                const int8_t d = (int8_t)(x & 0xff);
                if (d) used |= 1u << t;
                x = (x - d) >> 8;
            }
        }
    } else {
        used = 0xf;   // any int32: four digits
    }
    if (!used) used = 1;
    int S = 0;
    for (int t = 0; t < 8; t++)
        if (used & (1u << t)) dg->shift[S++] = 8 * t;
    for (int s = S; s < NE_MAX_DIGITS; s++) dg->shift[s] = 0;
    dg->S = S;
    dg->l = 0;
    dg->lo = lo;
    dg->hi = hi;
    return NE_OK;
}



}  // namespace

// the plan; with a workspace its tables are uploaded on s, from the pinned
// host buffer staging when one is given (a copy that never waits for the host)
static ne_status plan_batch(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, void* workspace,
                            int64_t workspace_bytes, void* staging, int64_t staging_bytes, ne_batch_info* info,
                            cudaStream_t s) {
    if (!info || (njobs > 0 && !jobs) || njobs < 0) return fail(NE_EINVAL, "ne_batch_plan: bad arguments");
    if (cfg.ctas_per_sm < 1 || cfg.ctas_per_sm > 4) return fail(NE_EINVAL, "ne_batch_plan: ctas_per_sm=%d", cfg.ctas_per_sm);
    if (cfg.order != NE_ORDER_JOB && cfg.order != NE_ORDER_LPT) return fail(NE_EINVAL, "ne_batch_plan: order=%d", cfg.order);
    if (cfg.cconv_blocks != 4 && cfg.cconv_blocks != 8 && cfg.cconv_blocks != 16)
        return fail(NE_EINVAL, "ne_batch_plan: cconv_blocks=%d", cfg.cconv_blocks);
    if (cfg.l_policy != NE_L_BYTE && cfg.l_policy != NE_L_SMALLEST)
        return fail(NE_EINVAL, "ne_batch_plan: l_policy=%d", cfg.l_policy);
    if (cfg.ntt_min_n < 0) return fail(NE_EINVAL, "ne_batch_plan: ntt_min_n=%d", cfg.ntt_min_n);
    std::vector<DevJob> dj((size_t)njobs);
    std::vector<NJob> nj;
    int64_t ntt_ws = 0, ntt_units = 0;
    int ntt_max_logL = 0, ntt_max_M = 0, ntt_min_logL = 31;
    // with a workspace the tile and segment lists are built (product tiles and
    // convolution tiles apart); without one only counted, for the sizes
    const bool build = workspace != nullptr;
    struct GemmJob {
        int32_t job, rt, ct;
        int64_t cost;            // of each of its tiles
    };
    std::vector<GemmJob> gjobs;
    std::vector<DevTile> tiles_c;
    std::vector<int64_t> cost_c;
    std::vector<DevSeg> segs;
    int64_t n_tiles_g = 0, n_tiles_c = 0, n_segs = 0;
    int64_t plane_bytes = 0, flag_words = 0, mma_ops = 0, useful = 0;
    for (int32_t i = 0; i < njobs; i++) {
        const ne_job& j = jobs[i];
        DevJob& d = dj[(size_t)i];
        std::memset(&d, 0, sizeof(d));
        if (j.kind != NE_JOB_GEMM && j.kind != NE_JOB_CCONV) return fail(NE_EINVAL, "job %d: kind %d", i, j.kind);
        if (j.M < 3 || j.M > 5) return fail(NE_EINVAL, "job %d: M=%d (batches take 3..5 streams)", i, j.M);
        if (j.fuse != NE_FUSE_EXTRACT_CHECK && j.fuse != NE_FUSE_RECOVER && j.fuse != NE_FUSE_NONE)
            return fail(NE_EINVAL, "job %d: fuse", i);
        if (j.plain != 0 && (j.plain != 1 || j.fuse != NE_FUSE_NONE))
            return fail(NE_EINVAL, "job %d: a plain job has no check or recovery (fuse must be NE_FUSE_NONE)", i);
        if (j.r < 0 || j.r >= j.M) return fail(NE_EINVAL, "job %d: r=%d", i, j.r);
        if (j.cmin > j.cmax) return fail(NE_EINVAL, "job %d: empty value range", i);
        if (j.c_off < 0 || j.c_off % 4 || j.op_off < 0 || j.out_off < 0 || j.flag_off < 0)
            return fail(NE_EINVAL, "job %d: offsets (c_off must be a multiple of 4)", i);
        if (j.fault_begin < 0 || j.fault_end < j.fault_begin) return fail(NE_EINVAL, "job %d: fault range", i);
        int64_t K;
        if (j.kind == NE_JOB_GEMM) {
            if (j.rows < 1 || j.cols < 1 || j.k < 1 || j.k > 131056)
                return fail(NE_EINVAL, "job %d: GEMM %dx%dx%d (1 <= k <= 131056)", i, j.rows, j.cols, j.k);
            if (j.op_off % 4) return fail(NE_EINVAL, "job %d: op_off must be a multiple of 4", i);
            K = j.k;
        } else {
            if (j.N < 2 || j.N > 65536) return fail(NE_EINVAL, "job %d: N=%d (2 <= N <= 65536)", i, j.N);
            if (j.op_off % 4) return fail(NE_EINVAL, "job %d: op_off must be a multiple of 4", i);
            K = j.N;
        }
        const int64_t amax = std::max((int64_t)std::abs((int64_t)j.cmin), (int64_t)std::abs((int64_t)j.cmax));
        const int64_t bound = K * amax * 128;
        int32_t l = j.l, kk = 0;
        ne_digits dg;
        ne_status st;
        if (j.plain) {
            // the raw streams: digits of the values themselves (no predecessor term)
            if ((st = plain_digits(j.cmin, j.cmax, &dg))) return fail(st, "job %d: digit plan", i);
            l = 0;
            if (!make_fast_plan(dg, 0, &d.fp)) return fail(NE_ERANGE, "job %d: values need digits above the fourth", i);
            d.fp.pmask = 0;
        } else {
            if (l == 0) {
                st = ne_choose_l(j.M, 64, bound, cfg.l_policy, &l, &kk);
                if (st) return fail(st, "job %d: no l covers the bound %lld", i, (long long)bound);
            }
            ne_params p{j.M, l, 64};
            if ((st = validate_params(p))) return fail(st, "job %d: l=%d", i, l);
            if ((st = ne_plan_digits(l, j.cmin, j.cmax, &dg))) return fail(st, "job %d: digit plan", i);
            if (!make_fast_plan(dg, l, &d.fp)) return fail(NE_ERANGE, "job %d: words need digits above the fourth", i);
        }
        if (j.M * dg.S > MS_MAX) return fail(NE_EINVAL, "job %d: M*S=%d > %d", i, j.M * dg.S, MS_MAX);
        d.kind = j.kind;
        d.M = j.M;
        d.l = l;
        d.S = dg.S;
        d.MS = j.M * dg.S;
        d.rows = j.rows;
        d.cols = j.cols;
        d.k = j.kind == NE_JOB_GEMM ? (j.k + 15) / 16 * 16 : j.k;
        d.kc = j.k;
        d.N = j.N;
        d.r = j.r;
        d.fuse = j.fuse;
        for (int t = 0; t < NE_MAX_DIGITS; t++) d.shift[t] = t < dg.S ? dg.shift[t] : 0;
        d.c_off = j.c_off;
        d.op_off = j.op_off;
        d.out_off = j.out_off;
        d.flag_off = j.flag_off;
        d.fault_begin = j.fault_begin;
        d.fault_end = j.fault_end;
        d.npos = j.kind == NE_JOB_GEMM ? (int64_t)j.rows * d.k : (int64_t)j.N;
        d.nout = j.kind == NE_JOB_GEMM ? (int64_t)j.rows * j.cols : (int64_t)j.N;
        flag_words = std::max(flag_words, j.flag_off + (d.nout + 31) / 32);
        const int32_t cabs = (int32_t)amax;
        // the tensor tiles take whole Toeplitz blocks of 64: any other length
        // runs on the exact transforms, as do lengths from ntt_min_n on
        const bool ragged_n = j.kind == NE_JOB_CCONV && j.N % cconv::T != 0;
        const bool exact = j.kind == NE_JOB_CCONV && ntt_any_exact(j.M, j.plain ? 0 : l, j.N, cabs, j.plain != 0);
        if (ragged_n && !exact)
            return fail(NE_ERANGE, "job %d: N=%d is not a multiple of 64 and its outputs leave the exact transforms' "
                                   "range", i, j.N);
        if (j.kind == NE_JOB_CCONV && exact && (ragged_n || (cfg.ntt_min_n > 0 && j.N >= cfg.ntt_min_n))) {
            // the exact transform path: no digit planes, segments or tiles
            NJob t;
            std::memset(&t, 0, sizeof(t));
            int lg = 0;
            t.L = ntt_any_length(j.N, &lg);
            t.logL = lg;
            t.c_off = j.c_off;
            t.g_off = j.op_off;
            t.out_off = j.out_off;
            t.flag_off = j.flag_off;
            t.ws_off = ntt_ws / 4;
            t.fault_begin = j.fault_begin;
            t.fault_end = j.fault_end;
            t.M = j.M;
            t.N = j.N;
            t.l = j.plain ? 0 : l;
            t.r = j.fuse == NE_FUSE_NONE ? 0 : j.r;
            t.fuse = j.fuse;
            t.plain = j.plain;
            t.lo = j.cmin;
            t.hi = j.cmax;
            ntt_any_job_constants(t);
            nj.push_back(t);
            ntt_ws = align256(ntt_ws + (int64_t)(j.M + 1) * 2 * t.L * 4);
            ntt_units = std::max(ntt_units, (int64_t)(j.M + 1) * t.L);
            ntt_max_logL = std::max(ntt_max_logL, lg);
            ntt_min_logL = std::min(ntt_min_logL, lg);
            ntt_max_M = std::max(ntt_max_M, (int)j.M);
            d.plane_off = plane_bytes;           // no planes
            useful += 2LL * j.M * j.N * j.N;
            continue;
        }
        d.plane_off = plane_bytes;
        plane_bytes = align256(plane_bytes + (int64_t)d.MS * d.npos);
        if (j.kind == NE_JOB_GEMM && d.k != d.kc) {
            // rows padded to 16: entangled row by row
            const int64_t rps = std::max<int64_t>(1, SEG / d.k);
            n_segs += (j.rows + rps - 1) / rps;
            if (build)
                for (int64_t r0 = 0; r0 < j.rows; r0 += rps)
                    segs.push_back(DevSeg{i, SEG_ROWS, r0, std::min<int64_t>(rps, j.rows - r0)});
        } else {
            n_segs += (d.npos + SEG - 1) / SEG;
            if (build)
                for (int64_t s0 = 0; s0 < d.npos; s0 += SEG)
                    segs.push_back(DevSeg{i, SEG_ENTANGLE, s0, std::min<int64_t>(SEG, d.npos - s0)});
        }
        if (j.kind == NE_JOB_GEMM) {
            d.gt_off = plane_bytes;
            plane_bytes = align256(plane_bytes + (int64_t)j.cols * d.k);
            const int64_t ntt = (int64_t)((d.k + TT - 1) / TT) * ((j.cols + TT - 1) / TT);
            n_segs += (ntt + TT_PER_SEG - 1) / TT_PER_SEG;
            const int rt = (j.rows + bgemm::BM - 1) / bgemm::BM, ct = (j.cols + bgemm::BN - 1) / bgemm::BN;
            n_tiles_g += (int64_t)rt * ct;
            if (build) {
                for (int64_t s0 = 0; s0 < ntt; s0 += TT_PER_SEG)
                    segs.push_back(DevSeg{i, SEG_TRANSPOSE, s0, std::min<int64_t>(TT_PER_SEG, ntt - s0)});
                gjobs.push_back(GemmJob{i, rt, ct, (int64_t)d.MS * bgemm::BM * bgemm::BN * d.k});
            }
            mma_ops += 2LL * d.MS * rt * bgemm::BM * ct * bgemm::BN * d.k;
            useful += 2LL * j.M * j.rows * j.cols * j.k;
        } else {
            const int NB = j.N / cconv::T;
            const int npb = std::min(cfg.cconv_blocks, NB);
            n_tiles_c += (NB + npb - 1) / npb;
            if (build)
                for (int a = 0; a * npb < NB; a++) {
                    tiles_c.push_back(DevTile{i, NE_JOB_CCONV, a, npb});
                    cost_c.push_back((int64_t)d.MS * std::min(npb, NB - a * npb) * cconv::T * j.N);
                }
            mma_ops += 2LL * d.MS * j.N * j.N;
            useful += 2LL * j.M * j.N * j.N;
        }
    }
    const int64_t ntiles = n_tiles_g + n_tiles_c, ngemm = n_tiles_g;
    if (ntiles > 0x7fffffff || n_segs > 0x7fffffff) return fail(NE_EINVAL, "ne_batch_plan: batch too large");
    if (nj.size() > 65535) return fail(NE_EINVAL, "ne_batch_plan: more than 65535 transform jobs");
    const Layout L = layout(njobs, ntiles, n_segs, plane_bytes, (int64_t)nj.size(), ntt_ws);
    info->njobs = njobs;
    info->ntiles = (int32_t)ntiles;
    info->ngemm_tiles = (int32_t)ngemm;
    info->gemm_grid = sm_count() * bgemm::CTAS;
    info->nsegs = (int32_t)n_segs;
    info->grid = sm_count() * cfg.ctas_per_sm;
    info->flag_words = flag_words;
    info->workspace_bytes = L.total;
    info->mma_ops = mma_ops;
    info->useful_ops = useful;
    info->ntransform = (int32_t)nj.size();
    info->ntt_max_logL = ntt_max_logL;
    info->ntt_max_M = ntt_max_M;
    info->ntt_min_logL = nj.empty() ? 0 : ntt_min_logL;
    info->ntt_table_off = L.ntt_table;
    info->ntt_ws_off = L.ntt_ws;
    info->ntt_units = ntt_units;
    info->table_bytes = L.planes + (int64_t)nj.size() * (int64_t)sizeof(NJob);
    if (!workspace) return NE_OK;
    if (staging && staging_bytes < info->table_bytes)
        return fail(NE_EINVAL, "ne_batch_plan: staging buffer of %lld bytes < %lld", (long long)staging_bytes,
                    (long long)info->table_bytes);
    if (!nj.empty()) {
        // the twiddle tables are filled here, outside any stream capture of the runs
        ne_status st = ntt_any_init_tables(s);
        if (st) return st;
    }
    if (workspace_bytes < L.total) return fail(NE_ENOMEM, "ne_batch_plan: workspace %lld < %lld bytes",
                                               (long long)workspace_bytes, (long long)L.total);
    if (!aligned(workspace, 256)) return fail(NE_EINVAL, "ne_batch_plan: workspace must be 256-byte aligned");
    std::vector<uint8_t> host_vec;
    uint8_t* host;
    if (staging) {
        host = static_cast<uint8_t*>(staging);
        std::memset(host, 0, (size_t)L.jobs);      // the counters (the gaps between tables are never read)
    } else {
        host_vec.assign((size_t)L.planes, 0);
        host = host_vec.data();
    }
    std::memcpy(host + L.jobs, dj.data(), dj.size() * sizeof(DevJob));
    // the product tiles first (their own launch), then the convolution tiles;
    // within each list job order, or the most costly first (stable; all tiles
    // of a product job cost the same, so its jobs are sorted instead)
    const bool lpt = cfg.order == NE_ORDER_LPT;
    DevTile* dst = reinterpret_cast<DevTile*>(host + L.tiles);
    if (lpt) std::stable_sort(gjobs.begin(), gjobs.end(), [](const GemmJob& x, const GemmJob& y) { return x.cost > y.cost; });
    for (const GemmJob& g : gjobs)
        for (int a = 0; a < g.rt; a++)
            for (int b = 0; b < g.ct; b++) *dst++ = DevTile{g.job, NE_JOB_GEMM, a, b};
    std::vector<uint32_t> idx(tiles_c.size());
    for (size_t t = 0; t < idx.size(); t++) idx[t] = (uint32_t)t;
    if (lpt) std::stable_sort(idx.begin(), idx.end(), [&](uint32_t x, uint32_t y) { return cost_c[x] > cost_c[y]; });
    for (size_t t = 0; t < idx.size(); t++) *dst++ = tiles_c[idx[t]];
    if (!segs.empty()) std::memcpy(host + L.segs, segs.data(), segs.size() * sizeof(DevSeg));
    const void* njsrc = nj.data();
    if (staging && !nj.empty()) {
        std::memcpy(host + L.planes, nj.data(), nj.size() * sizeof(NJob));
        njsrc = host + L.planes;
    }
    if (cudaMemcpyAsync(workspace, host, (size_t)L.planes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return check_launch("ne_batch_plan: copy tables");
    if (!nj.empty() && cudaMemcpyAsync(static_cast<uint8_t*>(workspace) + L.ntt_table, njsrc,
                                       nj.size() * sizeof(NJob), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return check_launch("ne_batch_plan: copy transform jobs");
    // no wait: a copy from pageable memory returns once its bytes are staged
    // (so the host vectors may go), one from the pinned staging buffer at once;
    // both are ordered on s before the runs
    return NE_OK;
}

extern "C" ne_status ne_batch_plan(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, void* workspace,
                                   int64_t workspace_bytes, ne_batch_info* info, cudaStream_t s) {
    return plan_batch(jobs, njobs, cfg, workspace, workspace_bytes, nullptr, 0, info, s);
}

extern "C" ne_status ne_batch_plan_staged(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, void* workspace,
                                          int64_t workspace_bytes, void* staging, int64_t staging_bytes,
                                          ne_batch_info* info, cudaStream_t s) {
    if (workspace && !staging) return fail(NE_EINVAL, "ne_batch_plan_staged: null staging buffer");
    return plan_batch(jobs, njobs, cfg, workspace, workspace_bytes, staging, staging_bytes, info, s);
}

extern "C" ne_status ne_batch_run(ne_batch_info info, const int32_t* c, const int8_t* ops, int64_t* out, uint32_t* flags,
                                  uint64_t* nflag, const int64_t* fault_pos, const int32_t* fault_stream,
                                  const int32_t* fault_bit, void* workspace, int32_t* status, cudaStream_t s) {
    if (!workspace || info.njobs < 0 || info.ntiles < 0 || info.grid < 1 || info.ngemm_tiles < 0 ||
        info.ngemm_tiles > info.ntiles || (info.ngemm_tiles > 0 && info.gemm_grid < 1))
        return fail(NE_EINVAL, "ne_batch_run: bad plan");
    if (info.njobs == 0) return NE_OK;
    if (!c || !ops || !out) return fail(NE_EINVAL, "ne_batch_run: null pointer");
    if ((fault_pos || fault_stream || fault_bit) && !(fault_pos && fault_stream && fault_bit))
        return fail(NE_EINVAL, "ne_batch_run: give all three fault lists or none");
    if (!aligned(c, 16) || !aligned(ops, 4) || !aligned(out, 8)) return fail(NE_EINVAL, "ne_batch_run: alignment");
    const Layout L = layout(info.njobs, info.ntiles, info.nsegs, 0);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    BatchK k;
    k.jobs = reinterpret_cast<const DevJob*>(ws + L.jobs);
    k.tiles = reinterpret_cast<const DevTile*>(ws + L.tiles);
    k.segs = reinterpret_cast<const DevSeg*>(ws + L.segs);
    k.counter = reinterpret_cast<int32_t*>(ws);
    k.planes = reinterpret_cast<int8_t*>(ws + L.planes);
    k.ngemm = info.ngemm_tiles;
    k.ntiles = info.ntiles;
    k.nsegs = info.nsegs;
    k.c = c;
    k.ops = ops;
    k.out = out;
    k.flags = flags;
    k.nflag = reinterpret_cast<unsigned long long*>(nflag);
    k.fault_pos = fault_pos;
    k.fault_stream = fault_stream;
    k.fault_bit = fault_bit;
    k.status = status;
    if (cudaMemsetAsync(k.counter, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return check_launch("ne_batch_run: counters");
    if (flags && info.flag_words > 0 && cudaMemsetAsync(flags, 0, (size_t)info.flag_words * 4, s) != cudaSuccess)
        return check_launch("ne_batch_run: flags");
    if (nflag && cudaMemsetAsync(nflag, 0, sizeof(uint64_t), s) != cudaSuccess) return check_launch("ne_batch_run: count");
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_batch_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bgemm::smem_bytes(MS_MAX)) != cudaSuccess ||
            cudaFuncSetAttribute(k_batch_cconv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cconv::smem_bytes(MS_MAX)) != cudaSuccess)
            return check_launch("ne_batch_run: shared-memory attribute");
        attr_set[dev] = true;
    }
    if (info.nsegs > 0) {
        int eg = std::min(info.nsegs, sm_count() * 8);
        k_batch_entangle<<<eg, THREADS, 0, s>>>(k);
        ne_status st = check_launch("ne_batch_run: entangle");
        if (st) return st;
    }
    if (info.ngemm_tiles > 0) {
        k_batch_gemm<<<info.gemm_grid, THREADS, bgemm::smem_bytes(MS_MAX), s>>>(k);
        ne_status st = check_launch("ne_batch_run: product tiles");
        if (st) return st;
    }
    if (info.ntiles > info.ngemm_tiles) {
        k_batch_cconv<<<info.grid, THREADS, cconv::smem_bytes(MS_MAX), s>>>(k);
        ne_status st = check_launch("ne_batch_run: convolution tiles");
        if (st) return st;
    }
    if (info.ntransform > 0) {
        NttAnyArgs a{};
        a.jobs.table = reinterpret_cast<const NJob*>(ws + info.ntt_table_off);
        a.jobs.njobs = info.ntransform;
        a.c = c;
        a.g = ops;
        a.out = out;
        a.flags = flags;
        a.nflag = reinterpret_cast<unsigned long long*>(nflag);
        a.flags_atomic = 1;
        a.status = status;
        a.ws = reinterpret_cast<uint32_t*>(ws + info.ntt_ws_off);
        a.fault_pos = fault_pos;
        a.fault_stream = fault_stream;
        a.fault_bit = fault_bit;
        return ntt_any_run(a, info.ntt_min_logL, info.ntt_max_logL, info.ntt_max_M, info.ntt_units, s);
    }
    return NE_OK;
}

// ---- the batch for callers that cannot allocate device memory ----------------------------------
//
// The scratch memory of a batch (plan tables and digit planes) lives in one
// static device array owned by the library instead of a caller workspace.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with that device current.

namespace {

__device__ __align__(256) uint8_t g_static_workspace[NE_STATIC_WORKSPACE_BYTES];
void* g_static_workspace_ptr[64] = {nullptr};   // per device, filled on first use

}  // namespace

extern "C" ne_status ne_batch_run_static(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, const int32_t* c,
                                         const int8_t* ops, int64_t* out, uint32_t* flags, uint64_t* nflag,
                                         const int64_t* fault_pos, const int32_t* fault_stream,
                                         const int32_t* fault_bit, int32_t* status, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(NE_ECUDA, "ne_batch_run_static: no usable current device");
    if (!g_static_workspace_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess || !p)
            return fail(NE_ECUDA, "ne_batch_run_static: address of the static workspace: %s", cudaGetErrorString(e));
        g_static_workspace_ptr[dev] = p;
    }
    ne_batch_info info;
    ne_status st = ne_batch_plan(jobs, njobs, cfg, nullptr, 0, &info, s);
    if (st) return st;
    if (info.workspace_bytes > NE_STATIC_WORKSPACE_BYTES)
        return fail(NE_ENOMEM,
                    "ne_batch_run_static: the batch needs %lld bytes of scratch; the static workspace holds %lld "
                    "(use ne_batch_plan/ne_batch_run with a workspace)",
                    (long long)info.workspace_bytes, (long long)NE_STATIC_WORKSPACE_BYTES);
    st = ne_batch_plan(jobs, njobs, cfg, g_static_workspace_ptr[dev], NE_STATIC_WORKSPACE_BYTES, &info, s);
    if (st) return st;
    return ne_batch_run(info, c, ops, out, flags, nflag, fault_pos, fault_stream, fault_bit,
                        g_static_workspace_ptr[dev], status, s);
}
