// Host restatement of the FP32 fixed-point arithmetic of the block kernels (apply_kernels.cuh,
// FxAcc): the split of a scaled product s into the integer pair (qh, ql) with
// qh 2^L + ql = rint(s), in its two forms (s given, or t = s 2^-L given), and the conversion
// of a total (hi word, lo word) back to FP32 by one FMA.  Plain IEEE binary32 arithmetic with
// round to nearest even (SSE on x86-64, no contraction), fmaf from the C library.
//
// usage: fixed_split <L> <samples> <seed>   prints "split <n> conv <n> exact <n>" on success,
// or the first failing case and exits 1.
#include <cinttypes>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

static const float kMagic = 12582912.0f;   // 1.5 * 2^23
static const int32_t kMagicBits = 0x4B400000;

static int32_t bits(float f) {
    int32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}
static float pow2f(int k) { return std::ldexp(1.0f, k); }

// s given (the kernels' add_scaled)
static void split_s(float s, int L, int32_t& qh, int32_t& ql) {
    const float t = s * pow2f(-L);
    const float th = t + kMagic;
    const float hf = th - kMagic;
    const float r = std::fmaf(-hf, pow2f(L), s);
    const float rl = r + kMagic;
    qh = bits(th) - kMagicBits;
    ql = bits(rl) - kMagicBits;
}

// t = s 2^-L given (the kernels' add_prescaled)
static void split_t(float t, int L, int32_t& qh, int32_t& ql) {
    const float th = t + kMagic;
    const float fr = t - (th - kMagic);
    const float tl = std::fmaf(fr, pow2f(L), kMagic);
    qh = bits(th) - kMagicBits;
    ql = bits(tl) - kMagicBits;
}

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const int L = std::atoi(argv[1]);
    const long n = std::atol(argv[2]);
    std::mt19937_64 rng(std::strtoull(argv[3], nullptr, 10));
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    long nsplit = 0, nconv = 0, nexact = 0;
    // 1. split: |s| < 2^(L + 22), magnitudes log-uniform from 2^-40, both signs, plus ties
    for (long i = 0; i < n; ++i) {
        float s;
        if (i % 4 == 3) {
            // an exact half-integer (a tie for the low part)
            const double m = std::floor(u01(rng) * std::ldexp(1.0, std::min(L + 21, 23))) + 0.5;
            s = (float)((i & 8) ? -m : m);
        } else {
            const double e = -40.0 + u01(rng) * (L + 22 + 40 - 0.01);
            s = (float)(std::ldexp(1.0, 0) * std::pow(2.0, e));
            if (i & 1) s = -s;
        }
        if (!(std::fabs(s) < std::ldexp(1.0f, L + 22))) continue;
        int32_t ah, al, bh, bl;
        split_s(s, L, ah, al);
        split_t(s * pow2f(-L), L, bh, bl);
        const int64_t q = ((int64_t)ah << L) + al;
        const int64_t want = (int64_t)std::nearbyint((double)s);   // round half to even
        if (ah != bh || al != bl || q != want || std::llabs(al) > (1ll << (L - 1))) {
            std::printf("split L=%d s=%.9g: (%d, %d) vs (%d, %d), q=%" PRId64 " want %" PRId64 "\n", L, s, ah, al, bh,
                        bl, q, want);
            return 1;
        }
        ++nsplit;
    }
    // 2. conversion of a total: |hi| < 2^22, |lo| <= 2^29; fmaf(hi, 2^L, lo) against the
    //    exact integer hi 2^L + lo rounded once to FP32
    for (long i = 0; i < n; ++i) {
        const int32_t hi = (int32_t)(u01(rng) * 8388606.0) - 4194303;
        const int lob = (int)(u01(rng) * 30.0);
        int32_t lo = (int32_t)(u01(rng) * std::ldexp(2.0, lob)) - (int32_t)std::ldexp(1.0, lob);
        if (i % 5 == 0) lo = -(hi << std::min(L, 7));   // cancellation
        const int64_t q = ((int64_t)hi << L) + lo;
        const float v = std::fmaf((float)hi, pow2f(L), (float)lo);
        const float ref = (float)(double)q;   // |q| < 2^52: the double is exact, one rounding
        const double err = std::fabs((double)v - (double)q);
        const double ulp = ref == 0.0f ? 0.0 : std::ldexp(1.0, std::ilogb(ref) - 23);
        if (err > 0.5 * ulp + 32.0) {
            std::printf("conv L=%d hi=%d lo=%d: %.9g vs %" PRId64 "\n", L, hi, lo, v, q);
            return 1;
        }
        if (std::llabs(lo) <= (1 << 24)) {
            if (v != ref) {
                std::printf("conv (exact lo) L=%d hi=%d lo=%d: %.9g vs %.9g\n", L, hi, lo, v, ref);
                return 1;
            }
            ++nexact;
        }
        ++nconv;
    }
    std::printf("split %ld conv %ld exact %ld\n", nsplit, nconv, nexact);
    return 0;
}
