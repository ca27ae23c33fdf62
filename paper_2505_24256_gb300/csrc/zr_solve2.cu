// zr_solve2.cu -- instances of the per-warp-chain solve kernel (zr_solve2.cuh)
// for its column-group widths.
#include "zr_solve2.cuh"

namespace zr {

namespace {
template <int CG>
int occ2() { return solve2_occupancy_t<CG, solve2_warps(CG)>(); }
template <int CG>
void run2(const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
  launch_solve2_t<CG, solve2_warps(CG)>(Ds, items, nitems, sms, M, st);
}
}  // namespace

#define ZR_SOLVE2_WIDTHS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(14) X(16)

int solve2_widths(int* out, int cap) {
  int n = 0;
#define ZR_W(cg) if (n < cap) out[n++] = cg;
  ZR_SOLVE2_WIDTHS(ZR_W)
#undef ZR_W
  return n;
}

int solve2_occupancy(int cg) {
  switch (cg) {
#define ZR_C(x) case x: return occ2<x>();
    ZR_SOLVE2_WIDTHS(ZR_C)
#undef ZR_C
    default: return 0;
  }
}

int solve2_roots_per_item(int cg) { return 32 * solve2_warps(cg); }

bool launch_b_solve2(int cg, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
  if (nitems <= 0) return true;
  switch (cg) {
#define ZR_L(x) case x: run2<x>(Ds, items, nitems, sms, M, st); return true;
    ZR_SOLVE2_WIDTHS(ZR_L)
#undef ZR_L
    default: return false;
  }
}

}  // namespace zr
