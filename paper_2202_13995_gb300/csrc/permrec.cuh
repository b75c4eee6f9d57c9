// Row-permutation record of a panel factorization (shared by the panel
// kernels).
#pragma once
#include "common.cuh"

namespace gb {

// Row-permutation record: slot s holds position pos[s] and the original
// position cur[s] of the row that now sits there.  Positions [base, lim) use
// slots [0, lim - base) directly; other positions are found through an
// open-addressing hash (key = position, value = slot).  One thread only.
struct PermRec {
  int* pos;
  int* cur;
  int* hkey;
  int* hval;
  int mask;
  int base, lim;
  int* cnt;
  __device__ __forceinline__ int slot(int p) const {
    if (p < lim) return p - base;
    unsigned b = ((unsigned)p * 2654435761u) & (unsigned)mask;
    while (true) {
      const int k = hkey[b];
      if (k == p) return hval[b];
      if (k < 0) {
        const int s = (*cnt)++;
        hkey[b] = p;
        hval[b] = s;
        pos[s] = p;
        cur[s] = p;
        return s;
      }
      b = (b + 1) & (unsigned)mask;
    }
  }
  __device__ __forceinline__ void swap_rows(int a, int p) const {  // positions a (direct) and p
    const int sa = slot(a), sb = slot(p);
    const int t = cur[sa];
    cur[sa] = cur[sb];
    cur[sb] = t;
  }
};

}  // namespace gb
