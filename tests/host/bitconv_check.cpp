// Host check of the mixed-precision conversions of kernels.cuh (exponent_of,
// f64_to_f32_shift, f32_to_f64_shift). The test harness pastes the functions'
// source where the marker line is, compiled for the host with bit-cast stand-ins
// for the CUDA intrinsics, and this program compares them with C's own
// conversions (round to nearest, ties to even):
// - f32_to_f64_shift(x, s) == ldexp((double)x, s) exactly for normal x; zero and
//   subnormal x give a zero of x's sign; Inf and NaN give NaN;
// - f64_to_f32_shift(x, s) == (float)ldexp(x, s) whenever that is a normal float;
//   results below the normal range give a zero of x's sign, results that would
//   overflow give +-FLT_MAX;
// - exponent_of(x) == ilogb(x) for positive normal x, 0 for 0.
// Prints "ok" or the first failure; exit status 0 on success.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

static inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
static inline unsigned __float_as_uint(float x) { unsigned r; std::memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned x) { float r; std::memcpy(&r, &x, 4); return r; }
#define __device__
#define __forceinline__ inline

// @EXTRACTED@

static int fails = 0;
static void fail(const char *what, double x, int s, double got, double want) {
    if (fails++ < 5) printf("%s: x=%.17g shift=%d got=%.17g want=%.17g\n", what, x, s, got, want);
}

static bool same_bits_f(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }

static void check_narrow(double x, int s) {
    const float got = f64_to_f32_shift(x, s);
    const double y = std::ldexp(x, s);
    const float c = (float)y;
    float want;
    if (std::fabs(y) < FLT_MIN) want = std::signbit(x) ? -0.0f : 0.0f;
    else if (std::isinf(c)) want = std::signbit(x) ? -FLT_MAX : FLT_MAX;
    else want = c;
    if (!same_bits_f(got, want)) fail("f64_to_f32_shift", x, s, got, want);
}

int main() {
    std::mt19937_64 rng(12345);
    // widening: exact for every normal float and shift
    for (int n = 0; n < 2000000; n++) {
        const unsigned b = (unsigned)rng();
        const float x = __uint_as_float(b);
        const int s = (int)(rng() % 121) - 60;
        const double got = f32_to_f64_shift(x, s);
        const int e = (b >> 23) & 0xff;
        if (e == 0) {
            if (got != 0.0 || std::signbit(got) != std::signbit(x)) fail("f32_to_f64_shift zero", x, s, got, 0.0);
        } else if (e == 0xff) {
            if (!std::isnan(got)) fail("f32_to_f64_shift inf/nan", x, s, got, NAN);
        } else if (got != std::ldexp((double)x, s)) {
            fail("f32_to_f64_shift", x, s, got, std::ldexp((double)x, s));
        }
    }
    // narrowing: random bit patterns over the exponents that land near and inside the float range
    for (int n = 0; n < 4000000; n++) {
        const unsigned long long m = rng() & 0xfffffffffffffULL;
        const int s = (int)(rng() % 121) - 60;
        const int fe = (int)(rng() % 270) - 8;            // target float exponent field, -8 .. 261
        const int e = fe - 127 + 1023 - s;
        if (e <= 0 || e >= 0x7ff) continue;
        const unsigned long long sign = (rng() & 1) << 63;
        const double x = __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | m));
        check_narrow(x, s);
    }
    // ties and carries: the dropped 29 bits exactly half, just below and just above
    for (unsigned long long keep : {0ULL, 1ULL, 2ULL, 0x3fffffULL, 0x7ffffeULL, 0x7fffffULL})
        for (unsigned long long rem : {0x0fffffffULL, 0x10000000ULL, 0x10000001ULL, 0x1fffffffULL, 0ULL})
            for (int fe : {1, 2, 127, 253, 254})
                for (int s : {-30, 0, 17}) {
                    const int e = fe - 127 + 1023 - s;
                    const double x = __longlong_as_double((long long)(((unsigned long long)e << 52) | (keep << 29) | rem));
                    check_narrow(x, s);
                    check_narrow(-x, s);
                }
    // special inputs
    check_narrow(0.0, 3);
    check_narrow(-0.0, -3);
    if (!same_bits_f(f64_to_f32_shift(INFINITY, 0), FLT_MAX)) fail("inf", INFINITY, 0, f64_to_f32_shift(INFINITY, 0), FLT_MAX);
    if (std::fabs(f64_to_f32_shift(NAN, 0)) != FLT_MAX) fail("nan", NAN, 0, f64_to_f32_shift(NAN, 0), FLT_MAX);
    // exponent_of
    for (int n = 0; n < 1000000; n++) {
        const unsigned long long b = rng() & 0x7fffffffffffffffULL;
        const double x = __longlong_as_double((long long)b);
        const int e = (int)(b >> 52);
        if (e == 0 || e == 0x7ff) continue;
        if (exponent_of(x) != std::ilogb(x)) fail("exponent_of", x, 0, exponent_of(x), std::ilogb(x));
    }
    if (exponent_of(0.0) != 0) fail("exponent_of(0)", 0.0, 0, exponent_of(0.0), 0);
    if (fails) { printf("%d failures\n", fails); return 1; }
    printf("ok\n");
    return 0;
}
