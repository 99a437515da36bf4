// Host check of the library's derive27 (8 counted cells + pair tables + marginals -> 27
// cells) against brute-force counting of random genotype triples.
#include <cstdio>
#include <cstdlib>
#include "../../paper_2201_10956_gb300/csrc/epi3_internal.cuh"
int main() {
  srand(1);
  for (int trial = 0; trial < 20000; ++trial) {
    int n = rand() % 300;
    int full[27] = {0};
    int gx[300], gy[300], gz[300];
    for (int s = 0; s < n; ++s) { gx[s] = rand() % 3; gy[s] = rand() % 3; gz[s] = rand() % 3; full[9*gx[s]+3*gy[s]+gz[s]]++; }
    int n8[8] = {0}; int xy[4] = {0}, xz[4] = {0}, yz[4] = {0}; int mx[2]={0}, my[2]={0}, mz[2]={0};
    for (int s = 0; s < n; ++s) {
      if (gx[s] < 2 && gy[s] < 2 && gz[s] < 2) n8[4*gx[s]+2*gy[s]+gz[s]]++;
      if (gx[s] < 2 && gy[s] < 2) xy[2*gx[s]+gy[s]]++;
      if (gx[s] < 2 && gz[s] < 2) xz[2*gx[s]+gz[s]]++;
      if (gy[s] < 2 && gz[s] < 2) yz[2*gy[s]+gz[s]]++;
      if (gx[s] < 2) mx[gx[s]]++; if (gy[s] < 2) my[gy[s]]++; if (gz[s] < 2) mz[gz[s]]++;
    }
    int r[27];
    epi3::derive27(n8, make_int4(xy[0],xy[1],xy[2],xy[3]), make_int4(xz[0],xz[1],xz[2],xz[3]), make_int4(yz[0],yz[1],yz[2],yz[3]),
                   make_int2(mx[0],mx[1]), make_int2(my[0],my[1]), make_int2(mz[0],mz[1]), n, r);
    for (int q = 0; q < 27; ++q) if (r[q] != full[q]) { printf("MISMATCH trial %d cell %d: %d vs %d\n", trial, q, r[q], full[q]); return 1; }
  }
  printf("derive27 ok\n");
  return 0;
}
