// Host check of the red-black split-row layout (kernels.cuh, Geom::pos, xm,
// xp, nhalf): every vertex of a sample has its own position inside the sample's
// extent; even x sits in the first half of its row and odd x in the second;
// xm / xp reach the x-neighbours and the row / plane pitches the y / z ones.
// The geometry is built with the half-row length rounded up to 32 elements, as
// the runtime builds it. Prints "ok" or the first failure; exit status 0 on success.
#include <cstdio>
#include <vector>
#include "../../paper_2608_00760_b300/csrc/kernels.cuh"

using namespace dmgk;

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

int main() {
    const int shapes[][3] = {{3, 3, 3}, {5, 9, 17}, {17, 5, 9}, {65, 3, 5}, {129, 7, 3}, {257, 5, 5}, {4, 6, 3}};
    for (const auto &s : shapes) {
        const Geom g = geom(s[0], s[1], s[2]);
        if (g.nhalf() != (g.nx + 1) / 2 || g.nhalf() > g.hx) { printf("nhalf %d\n", g.nx); return 1; }
        std::vector<char> seen((size_t)g.sb, 0);
        for (int k = 0; k < g.nz; k++)
            for (int j = 0; j < g.ny; j++)
                for (int i = 0; i < g.nx; i++) {
                    const long long p = g.pos(i, j, k);
                    if (p < 0 || p >= g.sb || seen[p]) { printf("pos %d %d %d of %dx%dx%d\n", i, j, k, g.nx, g.ny, g.nz); return 1; }
                    seen[p] = 1;
                    const long long row = (long long)k * g.sz + (long long)j * g.sy;
                    if ((i % 2 == 0) != (p - row < g.hx)) { printf("half %d\n", i); return 1; }
                    if (i > 0 && g.pos(i - 1, j, k) != p + g.xm(i)) { printf("xm %d\n", i); return 1; }
                    if (i < g.nx - 1 && g.pos(i + 1, j, k) != p + g.xp(i)) { printf("xp %d\n", i); return 1; }
                    if (j > 0 && g.pos(i, j - 1, k) != p - g.sy) { printf("y %d\n", j); return 1; }
                    if (k > 0 && g.pos(i, j, k - 1) != p - g.sz) { printf("z %d\n", k); return 1; }
                }
    }
    printf("ok\n");
    return 0;
}
