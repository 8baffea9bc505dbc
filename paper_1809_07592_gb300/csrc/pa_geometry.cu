// pa_geometry.cu -- choice of transform length and pass split.
//
// The cyclic length only has to cover the linear-convolution window, L >= n+m-1
// (paper Section 2.2: FFT length n+r-1). Restricting L to powers of two can
// almost double the work (n+m-1 just above 2^k); smooth lengths ro * 2^k with
// ro in {3, 5, 9} cut that padding, at the price of one odd-radix stage in the
// innermost pass.
#include <cmath>
#include <cstdlib>

#include "pa_internal.h"
#include "pa_launch.h"

namespace pa {

namespace {

int lg_max_inner(pa_dtype_t d, bool split) {
    if (split) return d == PA_FP32_GUARD ? MaxLgSplit<float>::v : MaxLgSplit<double>::v;
    return d == PA_FP32_GUARD ? MaxLgMiddle<float>::v : d == PA_FP64 ? MaxLgMiddle<double>::v : MaxLgMiddle<Zp>::v;
}

bool inner_valid(pa_dtype_t d, int ro, int lgI, bool split) {
    if (ro == 1) return lgI >= kMinLgMiddle && lgI <= lg_max_inner(d, split);
    if (d == PA_NTT64) return false;
    return d == PA_FP32_GUARD ? odd_inner_ok<float>(ro, lgI, split) : odd_inner_ok<double>(ro, lgI, split);
}

// L = ro * 2^k; returns false if L is not of that form.
bool decompose(uint64_t L, int *ro, int *k) {
    uint64_t o = L;
    int e = 0;
    while (o && !(o & 1)) {
        o >>= 1;
        ++e;
    }
    if (o != 1 && o != 3 && o != 5 && o != 9) return false;
    *ro = (int)o;
    *k = e;
    return true;
}

}  // namespace

std::vector<Geometry> geometry_candidates(uint64_t L, pa_dtype_t dtype, bool split) {
    std::vector<Geometry> two, three;
    int ro, k;
    if (!decompose(L, &ro, &k)) return two;
    for (int lg1 = kMinLgStrided; lg1 <= kMaxLgStrided; ++lg1) {
        const int lgI2 = k - lg1;
        if (lgI2 >= 0 && inner_valid(dtype, ro, lgI2, split)) two.push_back(Geometry{L, lg1, 0, ro, lgI2});
        for (int lgM = kMinLgStrided; lgM <= kMaxLgStrided; ++lgM) {
            const int lgI3 = k - lg1 - lgM;
            if (lgI3 >= 0 && inner_valid(dtype, ro, lgI3, split)) three.push_back(Geometry{L, lg1, lgM, ro, lgI3});
        }
    }
    return two.empty() ? three : two;
}

Geometry default_geometry(uint64_t L, pa_dtype_t dtype, bool split) {
    std::vector<Geometry> c = geometry_candidates(L, dtype, split);
    Geometry best;
    int bestd = 1 << 30;
    for (const Geometry &g : c) {
        // innermost length closest to 2^11.5 (measured sweet spot of one CTA's transform);
        // distances in units of 1/100 of a power of two, the first (larger inner) wins ties
        const int lg100 = (int)(100.0 * std::log2((double)g.inner()));
        const int d = lg100 > 1150 ? lg100 - 1150 : 1150 - lg100;
        if (d < bestd) {
            bestd = d;
            best = g;
        }
    }
    return best;
}

Geometry choose_geometry(uint64_t need, pa_dtype_t dtype, bool split) {
    if (need < 4096) need = 4096;
    Geometry best;
    const int ros[4] = {1, 3, 5, 9};
    const bool smooth = std::getenv("PA_POW2_ONLY") == nullptr;  // lets a user force powers of two
    for (int ro : ros) {
        if (ro > 1 && (dtype == PA_NTT64 || !smooth)) continue;
        for (int k = 0; k <= 28; ++k) {
            const uint64_t L = (uint64_t)ro << k;
            if (L > (1ull << 28)) break;
            if (L < need) continue;
            Geometry g = default_geometry(L, dtype, split);
            if (g.L == 0) continue;  // no valid split at this length: try the next
            if (best.L == 0 || g.L < best.L) best = g;
            break;
        }
    }
    return best;
}

}  // namespace pa
