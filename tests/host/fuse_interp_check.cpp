// Host check that the fused prolongation kernel forms each corrected neighbour
// value exactly as the separate prolongation does: for every fine vertex p, each
// of its six neighbours n, and random coarse corrections e, the value
// fuse_interp builds from p's coarse box equals, bit for bit, what prolong_cell
// adds at n. The functions' own source (kernels.cuh) is pasted where the marker
// line is. Box entries the kernel does not load are NaN here, so using one shows.
// Prints "ok" or the first failure; exit status 0 on success.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#define __host__
#define __device__
#define __forceinline__ inline
#define DMG_CHECK(cond)

// @EXTRACTED@

static Geom geom(int nx, int ny, int nz) {
    Geom g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.hx = (((nx + 1) / 2 + 31) / 32) * 32;
    g.sy = 2 * g.hx;
    g.sz = (long long)g.sy * ny;
    g.sb = g.sz * nz;
    g.nb = 1;
    return g;
}

static int fails = 0;

template <int PX, int PY, int PZ, int DX, int DY, int DZ>
static void check_one(const Geom &gc, const float *e, const Geom &gf, const float *P, int i, int j, int k) {
    const int I = (i >> 1) - 1, J = (j >> 1) - 1, K = (k >> 1) - 1;
    float B[3][3][3];
    for (int z = 0; z < 3; z++)
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++)
                B[z][y][x] = fuse_needed(PX, PY, PZ, x - 1, y - 1, z - 1) ? e[gc.pos(I + x, J + y, K + z)] : NAN;
    const float v = fuse_interp<PX, PY, PZ, DX, DY, DZ>(B);
    const float want = P[gf.pos(i + DX, j + DY, k + DZ)];
    if (!(v == want)) {
        if (fails++ < 5) printf("p=(%d,%d,%d) d=(%d,%d,%d): fused %.9g, prolong_cell %.9g\n", i, j, k, DX, DY, DZ, v, want);
    }
}

template <int PX, int PY, int PZ>
static void check_point(const Geom &gc, const float *e, const Geom &gf, const float *P, int i, int j, int k) {
    check_one<PX, PY, PZ, -1, 0, 0>(gc, e, gf, P, i, j, k);
    check_one<PX, PY, PZ, 1, 0, 0>(gc, e, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, -1, 0>(gc, e, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 1, 0>(gc, e, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 0, -1>(gc, e, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 0, 1>(gc, e, gf, P, i, j, k);
}

int main() {
    const int shapes[][3] = {{17, 9, 13}, {9, 17, 5}, {5, 5, 33}};
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> U(-1.0f, 1.0f);
    for (const auto &s : shapes)
        for (int trial = 0; trial < 3; trial++) {
            const Geom gf = geom(s[0], s[1], s[2]);
            const Geom gc = geom((s[0] - 1) / 2 + 1, (s[1] - 1) / 2 + 1, (s[2] - 1) / 2 + 1);
            std::vector<float> e((size_t)gc.sb, 0.0f), P((size_t)gf.sb, 0.0f);
            for (int K = 1; K < gc.nz - 1; K++)
                for (int J = 1; J < gc.ny - 1; J++)
                    for (int I = 1; I < gc.nx - 1; I++) {
                        float v = U(rng);
                        if (trial == 1) v = std::ldexp(std::round(8 * v), -3);   // exact sums and halvings
                        if (trial == 2) v = (I + J + K) % 3 ? v : 1e-30f;      // tiny values beside large ones
                        e[gc.pos(I, J, K)] = v;
                    }
            // the separate prolongation onto a zero fine array: one call per coarse cell
            for (int K = 0; K < gc.nz - 1; K++)
                for (int J = 0; J < gc.ny - 1; J++)
                    for (int I = 0; I < gc.nx - 1; I++) prolong_cell(gc, e.data(), gf, P.data(), I, J, K);
            for (int k = 1; k < gf.nz - 1; k++)
                for (int j = 1; j < gf.ny - 1; j++)
                    for (int i = 1; i < gf.nx - 1; i++) {
                        switch ((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) {
                        case 0: check_point<0, 0, 0>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 1: check_point<1, 0, 0>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 2: check_point<0, 1, 0>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 3: check_point<1, 1, 0>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 4: check_point<0, 0, 1>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 5: check_point<1, 0, 1>(gc, e.data(), gf, P.data(), i, j, k); break;
                        case 6: check_point<0, 1, 1>(gc, e.data(), gf, P.data(), i, j, k); break;
                        default: check_point<1, 1, 1>(gc, e.data(), gf, P.data(), i, j, k); break;
                        }
                    }
        }
    if (fails) { printf("%d failures\n", fails); return 1; }
    printf("ok\n");
    return 0;
}
