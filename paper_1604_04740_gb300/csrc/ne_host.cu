// Host-only parts of the C ABI: parameter planning (Eq. 13, Eq. 14, Table II),
// digit planning, error strings.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "ne_common.cuh"

namespace {
thread_local char g_msg[512] = "";
int g_sms[64] = {0};
}  // namespace

namespace ne {

ne_status fail(ne_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

ne_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(NE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return NE_OK;
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_sms[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        g_sms[dev] = v;
    }
    return g_sms[dev];
}

ne_status validate_params(const ne_params& p) {
    if (p.w != 64) return fail(NE_EINVAL, "w must be 64 (got %d)", p.w);
    if (p.M < 3 || p.M > 32) return fail(NE_EINVAL, "M must be in [3, 32] (got %d)", p.M);
    if (p.l < 1) return fail(NE_EINVAL, "l must be >= 1 (got %d)", p.l);
    // Eq. 13 with k >= 1: (M-1) l <= w - 1
    if ((int64_t)(p.M - 1) * p.l > 63)
        return fail(NE_ERANGE, "(M-1)*l = %d violates Eq. 13 for w = 64", (p.M - 1) * p.l);
    return NE_OK;
}

ne_status validate_digits(const ne_digits& dg) {
    if (dg.S < 1 || dg.S > NE_MAX_DIGITS) return fail(NE_EINVAL, "digit count S = %d", dg.S);
    for (int s = 0; s < dg.S; s++) {
        if (dg.shift[s] % 8 != 0 || dg.shift[s] < 0 || dg.shift[s] > 56)
            return fail(NE_EINVAL, "digit shift %d is not a multiple of 8 in [0, 56]", dg.shift[s]);
        if (s > 0 && dg.shift[s] <= dg.shift[s - 1])
            return fail(NE_EINVAL, "digit shifts must be ascending");
    }
    return NE_OK;
}

ne_status validate_faults(const ne_faults& f, const char* who) {
    if (f.count < 0) return fail(NE_EINVAL, "%s: fault count %lld < 0", who, (long long)f.count);
    if (f.count > 0 && (!f.pos || !f.stream || !f.bit)) return fail(NE_EINVAL, "%s: null fault list", who);
    return NE_OK;
}

}  // namespace ne

using namespace ne;

namespace {
// Eq. 14 bound 2^((M-3)l+k) (2^(l-1)-1) as long double-free exact test:
// returns true when the bound is >= out_bound.
bool eq14_covers(int M, int l, int k, int64_t out_bound) {
    int e = (M - 3) * l + k;
    if (e < 0) return false;
    if (e + l >= 126) return true;
    unsigned __int128 D = ((unsigned __int128)1 << e) * (((unsigned __int128)1 << (l - 1)) - 1);
    return out_bound <= 0 || D >= (unsigned __int128)out_bound;
}
}  // namespace

extern "C" ne_status ne_choose_l(int32_t M, int32_t w, int64_t out_bound, int32_t policy,
                                 int32_t* l_out, int32_t* k_out) {
    if (!l_out || !k_out) return fail(NE_EINVAL, "ne_choose_l: null output pointer");
    if (M < 3 || w < 4 || w > 64) return fail(NE_EINVAL, "ne_choose_l: M=%d w=%d", M, w);
    if (policy == NE_L_PAPER) {
        int bl = -1, bk = -1, bv = -1, bt = -1;
        for (int l = 1; l < w; l++)
            for (int k = 1; k <= l; k++) {
                int t = (M - 1) * l + k;
                if (t > w) continue;
                int v = (M - 2) * l + k;
                if (v > bv || (v == bv && t > bt)) { bv = v; bt = t; bl = l; bk = k; }
            }
        if (bl < 0) return fail(NE_ERANGE, "ne_choose_l: no (l, k) for M=%d w=%d", M, w);
        *l_out = bl; *k_out = bk;
        return NE_OK;
    }
    if (policy == NE_L_SMALLEST || policy == NE_L_BYTE) {
        for (int l = 1; l < w; l++) {
            if (policy == NE_L_BYTE && l % 8) continue;
            for (int k = 1; k <= l && (M - 1) * l + k <= w; k++)
                if (eq14_covers(M, l, k, out_bound)) { *l_out = l; *k_out = k; return NE_OK; }
        }
        return fail(NE_ERANGE, "ne_choose_l: no l covers bound %lld for M=%d", (long long)out_bound, M);
    }
    return fail(NE_EINVAL, "ne_choose_l: unknown policy %d", policy);
}

static ne_status plan_digits_uncached(int32_t l, int32_t cmin, int32_t cmax, ne_digits* dg);

namespace {
// recent plans of this host thread (the enumeration below costs ~10^5 steps)
struct PlanCacheEntry {
    int32_t l, lo, hi;
    ne_digits dg;
    bool valid;
};
thread_local PlanCacheEntry g_plan_cache[16] = {};
thread_local int g_plan_next = 0;
}  // namespace

extern "C" ne_status ne_plan_digits(int32_t l, int32_t cmin, int32_t cmax, ne_digits* dg) {
    if (!dg) return fail(NE_EINVAL, "ne_plan_digits: null output");
    if (l < 1 || l > 62 || cmin > cmax) return fail(NE_EINVAL, "ne_plan_digits: l=%d range [%d, %d]", l, cmin, cmax);
    for (const PlanCacheEntry& e : g_plan_cache)
        if (e.valid && e.l == l && e.lo == cmin && e.hi == cmax) {
            *dg = e.dg;
            return NE_OK;
        }
    ne_status st = plan_digits_uncached(l, cmin, cmax, dg);
    if (st == NE_OK) {
        g_plan_cache[g_plan_next] = PlanCacheEntry{l, cmin, cmax, *dg, true};
        g_plan_next = (g_plan_next + 1) % 16;
    }
    return st;
}

static ne_status plan_digits_uncached(int32_t l, int32_t cmin, int32_t cmax, ne_digits* dg) {
    uint32_t used = 0;   // bit s set: digit s (weight 2^(8s)) can be non-zero
    int64_t span = (int64_t)cmax - cmin + 1;
    if (span <= 4096) {
        // enumerate every word eps = a + 2^l b with a, b in [cmin, cmax]
        for (int64_t a = cmin; a <= cmax; a++)
            for (int64_t b = cmin; b <= cmax; b++) {
                int64_t x = a + (int64_t)((uint64_t)b << l);
                for (int s = 0; s < 8 && x != 0; s++) {
                    int8_t d = (int8_t)(x & 0xff);      // balanced digit in [-128, 127]
                    if (d) used |= 1u << s;
                    x = (x - d) >> 8;                    // exact: x - d is a multiple of 256
                }
            }
        if (used == 0) used = 1;                         // all-zero data: keep one plane
    } else {
        // wide ranges: every digit up to the width of |eps| < amax (2^l + 1)
        int64_t amax = cmax > -(int64_t)cmin ? cmax : -(int64_t)cmin;
        int bits = 1;
        while (bits < 62 && ((int64_t)1 << bits) <= amax) bits++;
        int nd = (bits + l + 2 + 7) / 8;
        if (nd > NE_MAX_DIGITS) return fail(NE_ERANGE, "ne_plan_digits: %d digits needed", nd);
        used = (1u << nd) - 1;
    }
    int S = 0;
    for (int s = 0; s < 8; s++)
        if (used & (1u << s)) {
            if (S >= NE_MAX_DIGITS) return fail(NE_ERANGE, "too many digits");
            dg->shift[S++] = 8 * s;
        }
    for (int s = S; s < NE_MAX_DIGITS; s++) dg->shift[s] = 0;
    dg->S = S;
    dg->l = l;
    dg->lo = cmin;
    dg->hi = cmax;
    return NE_OK;
}

extern "C" const char* ne_last_error(void) { return g_msg; }

extern "C" const char* ne_version(void) { return "ne-gb300 0.1 (sm_103a)"; }
