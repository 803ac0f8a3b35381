// Host check of the batch split of blockIdx.z: the runtime's geometry
// (make_geom, dmg.cu) and the kernels' zsplit (kernels.cuh), their own source
// pasted where the marker line is, with host stand-ins for blockIdx and
// __umulhi. For every plane count d = nz - 2 + which and every z below the
// grid limit that a batch of nb samples launches (nb * d <= 65535), zsplit
// must return z / d as the sample and z mod d as the plane.
// Prints "ok" or the first failure; exit status 0 on success.
#include <cstdio>

static inline unsigned __umulhi(unsigned a, unsigned b) {
    return (unsigned)(((unsigned long long)a * (unsigned long long)b) >> 32);
}
static struct { unsigned x, y, z; } blockIdx;
#define __host__
#define __device__
#define __forceinline__ inline
#define DMG_CHECK(cond)

// @EXTRACTED@

int main() {
    for (int nz = 3; nz <= 4099; nz += (nz < 300 ? 1 : 17)) {
        for (int which = 0; which < 3; which++) {
            const int d = nz - 2 + which;
            const int nb = 65535 / d;
            const Geom g = make_geom(5, 5, nz, nb);
            for (unsigned z = 0; z < (unsigned)(nb * d); z++) {
                blockIdx.z = z;
                int plane;
                const int smp = zsplit(g, which, plane);
                if (smp != (int)(z / d) || plane != (int)(z % d)) {
                    printf("zsplit nz=%d which=%d z=%u -> %d %d\n", nz, which, z, smp, plane);
                    return 1;
                }
            }
        }
    }
    printf("ok\n");
    return 0;
}
