// Host check of the fused prolongation kernel's coarse-value box (kernels.cuh,
// fuse_lo / fuse_odd / fuse_needed). For a fine vertex with parities
// (px, py, pz), the six neighbours' trilinear interpolations (Eq. 17) weight
// the coarse vertices c with |2c - n| <= 1 per axis, n the neighbour's fine
// index. The box entries the kernel loads must be exactly the union of those
// supports, and each neighbour's (lo, odd) pair must describe its own support.
// Prints "ok" or the first mismatch; exit status 0 on success.
#include <cstdio>
#include "../../paper_2608_00760_b300/csrc/kernels.cuh"

using namespace dmgk;

int main() {
    const int D[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    int bad = 0;
    for (int pat = 0; pat < 8; pat++) {
        const int p[3] = {pat & 1, (pat >> 1) & 1, (pat >> 2) & 1};
        // fine index of the updated vertex along each axis: 2 * 5 + parity (any
        // base works; offsets are relative to base = fine >> 1 = 5)
        bool want[3][3][3] = {};
        for (int q = 0; q < 6; q++) {
            int n[3];
            for (int a = 0; a < 3; a++) n[a] = 10 + p[a] + D[q][a];
            for (int z = -1; z <= 1; z++)
                for (int y = -1; y <= 1; y++)
                    for (int x = -1; x <= 1; x++) {
                        const int c[3] = {5 + x, 5 + y, 5 + z};
                        bool w = true;
                        for (int a = 0; a < 3; a++) {
                            const int d = 2 * c[a] - n[a];
                            w = w && d >= -1 && d <= 1;
                        }
                        if (w) want[z + 1][y + 1][x + 1] = true;
                        // the neighbour's own support from (lo, odd)
                        bool mine = true;
                        const int r[3] = {x, y, z};
                        for (int a = 0; a < 3; a++) {
                            const int lo = fuse_lo(p[a], D[q][a]), od = fuse_odd(p[a], D[q][a]);
                            mine = mine && (r[a] == lo || (od && r[a] == lo + 1));
                        }
                        if (mine != w) {
                            if (!bad) printf("support mismatch: pattern %d neighbour %d entry (%d,%d,%d)\n", pat, q, x, y, z);
                            bad++;
                        }
                    }
        }
        for (int z = 0; z < 3; z++)
            for (int y = 0; y < 3; y++)
                for (int x = 0; x < 3; x++)
                    if (fuse_needed(p[0], p[1], p[2], x - 1, y - 1, z - 1) != want[z][y][x]) {
                        if (!bad) printf("box mismatch: pattern %d entry (%d,%d,%d)\n", pat, x - 1, y - 1, z - 1);
                        bad++;
                    }
    }
    if (bad) return 1;
    printf("ok\n");
    return 0;
}
