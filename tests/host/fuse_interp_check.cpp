// Host check that the prolongation kernels form each corrected value exactly as
// the separate prolongation does. The kernels take pairs of fine vertices
// i0 = 2m + par and i0 + 2 (m even) with one coarse box B[3][3][4] of x entries
// m-1 .. m+2. For every such pair, random coarse corrections e, and each
// vertex V of the pair that is interior:
//  - k_prolong_smooth32: the value fuse_interp builds for each of V's six
//    neighbours n equals, bit for bit, what prolong_cell adds at n;
//  - k_prolong_colour32: the value it builds for V itself (displacement 0)
//    equals what prolong_cell adds at V.
// The boxes hold exactly the entries the kernels load (needed by an interior
// vertex of the pair); the others are NaN here, so using one shows. The
// functions' own source (kernels.cuh) is pasted where the marker line is.
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

template <int PX, int PY, int PZ, int DX, int DY, int DZ, int V>
static void check_one(const float (&B)[3][3][4], const Geom &gf, const float *P, int i, int j, int k) {
    const float v = fuse_interp<PX, PY, PZ, DX, DY, DZ, V>(B);
    const float want = P[gf.pos(i + DX, j + DY, k + DZ)];
    if (!(v == want)) {
        if (fails++ < 5)
            printf("p=(%d,%d,%d) d=(%d,%d,%d) V=%d: fused %.9g, prolong_cell %.9g\n", i, j, k, DX, DY, DZ, V, v,
                   want);
    }
}

template <int PX, int PY, int PZ, int V>
static void check_vertex(const float (&Bs)[3][3][4], const float (&Bc)[3][3][4], const Geom &gf, const float *P,
                         int i, int j, int k) {
    check_one<PX, PY, PZ, -1, 0, 0, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 1, 0, 0, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, -1, 0, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 1, 0, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 0, -1, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 0, 1, V>(Bs, gf, P, i, j, k);
    check_one<PX, PY, PZ, 0, 0, 0, V>(Bc, gf, P, i, j, k);
}

// the pair starting at fine vertex i0 (parity PX) of row (j, k)
template <int PX, int PY, int PZ>
static void check_pair(const Geom &gc, const float *e, const Geom &gf, const float *P, int i0, int j, int k) {
    const bool v0 = i0 >= 1 && i0 <= gf.nx - 2, v1 = i0 + 2 <= gf.nx - 2;
    if (!v0 && !v1) return;
    const int I = (i0 >> 1) - 1, J = (j >> 1) - 1, K = (k >> 1) - 1;
    float Bs[3][3][4], Bc[3][3][4];
    for (int z = 0; z < 3; z++)
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 4; x++) {
                const bool ls = (v0 && fuse_needed_first(PX, PY, PZ, x, y, z)) ||
                                (v1 && fuse_needed_second(PX, PY, PZ, x, y, z));
                const bool lc = (v0 && x <= 2 && fuse_uses(PX, PY, PZ, 0, 0, 0, x - 1, y - 1, z - 1)) ||
                                (v1 && x >= 1 && fuse_uses(PX, PY, PZ, 0, 0, 0, x - 2, y - 1, z - 1));
                const float val = e[gc.pos(I + x, J + y, K + z)];
                Bs[z][y][x] = ls ? val : NAN;
                Bc[z][y][x] = lc ? val : NAN;
            }
    if (v0) check_vertex<PX, PY, PZ, 0>(Bs, Bc, gf, P, i0, j, k);
    if (v1) check_vertex<PX, PY, PZ, 1>(Bs, Bc, gf, P, i0 + 2, j, k);
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
                    for (int i0 = 0; i0 < gf.nx; i0++) {
                        if ((i0 >> 1) & 1) continue;   // pairs start at element m = i0 >> 1 even
                        switch ((i0 & 1) | ((j & 1) << 1) | ((k & 1) << 2)) {
                        case 0: check_pair<0, 0, 0>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 1: check_pair<1, 0, 0>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 2: check_pair<0, 1, 0>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 3: check_pair<1, 1, 0>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 4: check_pair<0, 0, 1>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 5: check_pair<1, 0, 1>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        case 6: check_pair<0, 1, 1>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        default: check_pair<1, 1, 1>(gc, e.data(), gf, P.data(), i0, j, k); break;
                        }
                    }
        }
    if (fails) { printf("%d failures\n", fails); return 1; }
    printf("ok\n");
    return 0;
}
