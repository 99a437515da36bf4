// Host check of the compacted tensor scan's derived first-SNP genotype (the library's cmp_geno,
// cmp_drop, relabel_xy, relabel_marg, relabel_xz and canon_rows): for random genotype triples
// of two classes and every choice d of the derived genotype, the cells counted for the two
// other genotypes of X plus the relabelled pair tables and marginals give, through derive27 and
// canon_rows, exactly the brute-force 27-cell tables of both classes; relabel_xz is relabel_xy
// in the tensor scan's +3 / +9 offsets; cmp_drop names the most frequent genotype over both
// classes.
#include <cstdio>
#include <cstdlib>
#include "../../paper_2201_10956_gb300/csrc/epi3_internal.cuh"

struct ClassTables {
    int full[27];
    int xy[4], xz[4], yz[4], mx[2], my[2], mz[2], gx_count[3];
    int n;
};

static void count(const int* gx, const int* gy, const int* gz, int n, ClassTables& t) {
    for (int q = 0; q < 27; ++q) t.full[q] = 0;
    for (int q = 0; q < 4; ++q) t.xy[q] = t.xz[q] = t.yz[q] = 0;
    for (int q = 0; q < 2; ++q) t.mx[q] = t.my[q] = t.mz[q] = 0;
    for (int q = 0; q < 3; ++q) t.gx_count[q] = 0;
    t.n = n;
    for (int s = 0; s < n; ++s) {
        t.full[9 * gx[s] + 3 * gy[s] + gz[s]]++;
        t.gx_count[gx[s]]++;
        if (gx[s] < 2 && gy[s] < 2) t.xy[2 * gx[s] + gy[s]]++;
        if (gx[s] < 2 && gz[s] < 2) t.xz[2 * gx[s] + gz[s]]++;
        if (gy[s] < 2 && gz[s] < 2) t.yz[2 * gy[s] + gz[s]]++;
        if (gx[s] < 2) t.mx[gx[s]]++;
        if (gy[s] < 2) t.my[gy[s]]++;
        if (gz[s] < 2) t.mz[gz[s]]++;
    }
}

int main() {
    srand(7);
    for (int trial = 0; trial < 20000; ++trial) {
        ClassTables cls[2];
        int gxs[2][300], gys[2][300], gzs[2][300];
        for (int c = 0; c < 2; ++c) {
            const int n = rand() % 300;
            // skewed genotype frequencies so that every genotype is sometimes the most frequent
            const int w0 = 1 + rand() % 6, w1 = 1 + rand() % 6, w2 = 1 + rand() % 6;
            for (int s = 0; s < n; ++s) {
                const int u = rand() % (w0 + w1 + w2);
                gxs[c][s] = u < w0 ? 0 : u < w0 + w1 ? 1 : 2;
                gys[c][s] = rand() % 3;
                gzs[c][s] = rand() % 3;
            }
            count(gxs[c], gys[c], gzs[c], n, cls[c]);
        }
        const int tot[3] = {cls[0].gx_count[0] + cls[1].gx_count[0], cls[0].gx_count[1] + cls[1].gx_count[1],
                            cls[0].gx_count[2] + cls[1].gx_count[2]};
        const int dd = epi3::cmp_drop(tot[0], tot[1], tot[2]);
        if (tot[dd] < tot[0] || tot[dd] < tot[1] || tot[dd] < tot[2]) {
            printf("cmp_drop %d is not a most frequent genotype (%d %d %d)\n", dd, tot[0], tot[1], tot[2]);
            return 1;
        }
        for (int d = 0; d < 3; ++d) {
            if (epi3::cmp_geno(d, 0) == d || epi3::cmp_geno(d, 1) == d ||
                epi3::cmp_geno(d, 0) >= epi3::cmp_geno(d, 1)) {
                printf("cmp_geno(%d) does not list the two other genotypes in order\n", d);
                return 1;
            }
            for (int c = 0; c < 2; ++c) {
                const ClassTables& t = cls[c];
                // the counted cells: slot s holds first-SNP genotype cmp_geno(d, s)
                int n8[8] = {0};
                for (int s = 0; s < t.n; ++s)
                    for (int slot = 0; slot < 2; ++slot)
                        if (gxs[c][s] == epi3::cmp_geno(d, slot) && gys[c][s] < 2 && gzs[c][s] < 2)
                            n8[4 * slot + 2 * gys[c][s] + gzs[c][s]]++;
                const int4 pxy = make_int4(t.xy[0], t.xy[1], t.xy[2], t.xy[3]);
                const int4 pxz = make_int4(t.xz[0], t.xz[1], t.xz[2], t.xz[3]);
                const int4 pyz = make_int4(t.yz[0], t.yz[1], t.yz[2], t.yz[3]);
                const int2 mx = make_int2(t.mx[0], t.mx[1]), my = make_int2(t.my[0], t.my[1]);
                const int2 mz = make_int2(t.mz[0], t.mz[1]);
                const int4 rxz = epi3::relabel_xy(pxz, mz, d);
                int r[27];
                epi3::derive27(n8, epi3::relabel_xy(pxy, my, d), rxz, pyz, epi3::relabel_marg(mx, t.n, d),
                               my, mz, t.n, r);
                epi3::canon_rows(r, d);
                for (int q = 0; q < 27; ++q)
                    if (r[q] != t.full[q]) {
                        printf("MISMATCH trial %d d %d class %d cell %d: %d vs %d\n", trial, d, c, q, r[q],
                               t.full[q]);
                        return 1;
                    }
                // the FP32 form with the tensor scan's offsets
                const float4 f = epi3::relabel_xz(make_float4(pxz.x + 3.f, pxz.y + 3.f, pxz.z + 3.f, pxz.w + 3.f),
                                                  make_float2(mz.x + 9.f, mz.y + 9.f), d);
                if (f.x != rxz.x + 3.f || f.y != rxz.y + 3.f || f.z != rxz.z + 3.f || f.w != rxz.w + 3.f) {
                    printf("relabel_xz differs from relabel_xy + 3 (trial %d, d %d)\n", trial, d);
                    return 1;
                }
            }
        }
    }
    printf("relabel ok\n");
    return 0;
}
