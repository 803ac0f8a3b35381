// Host check of the single-CTA tail's index decoding: the host's magic divisor
// (magic_div, dmg.cu) and the kernel's one-multiply division and (i, j, k)
// decode (mdiv, tail_decode, kernels.cuh), pasted where the marker line is with
// a host stand-in for __umulhi. For every divisor the tail uses (grid extents
// up to 4098) and every index it can see (below 2^16), mdiv must equal integer
// division and tail_decode must equal (t mod a, (t / a) mod b, t / (a b)).
// Prints "ok" or the first failure; exit status 0 on success.
#include <cstdio>

static inline unsigned __umulhi(unsigned a, unsigned b) {
    return (unsigned)(((unsigned long long)a * (unsigned long long)b) >> 32);
}
#define __device__
#define __forceinline__ inline
#define DMG_CHECK(cond)

// @EXTRACTED@

int main() {
    for (int d = 1; d <= 4098; d++) {
        const unsigned m = magic_div(d);
        const int step = d < 300 ? 1 : 7;
        for (int t = 0; t < 65536; t += step)
            if (mdiv(t, m) != t / d) { printf("mdiv t=%d d=%d got %d\n", t, d, mdiv(t, m)); return 1; }
        if (mdiv(65535, m) != 65535 / d) { printf("mdiv 65535 d=%d\n", d); return 1; }
    }
    const int dims[][2] = {{1, 1}, {1, 15}, {15, 15}, {7, 64}, {17, 3}, {64, 64}, {255, 7}, {4096, 1}, {2, 4098}};
    for (const auto &ab : dims) {
        const int a = ab[0], b = ab[1];
        for (int t = 0; t < 65536; t++) {
            int i, j, k;
            tail_decode(t, a, magic_div(a), b, magic_div(b), i, j, k);
            if (i != t % a || j != (t / a) % b || k != t / (a * b)) {
                printf("tail_decode t=%d a=%d b=%d -> %d %d %d\n", t, a, b, i, j, k);
                return 1;
            }
        }
    }
    printf("ok\n");
    return 0;
}
