// zr_solve_narrow.cu -- solve instances with 2 and 3 right-hand sides per
// consumer thread (every consumer-warp count).
#include "zr_solve.cuh"

namespace zr {

int solve_occupancy_narrow(int cg, int g) {
  if (cg == 2) return SolveTile<2, 1>::exists(g) ? SolveTile<2, 1>::occupancy(g) : 0;
  if (cg == 3) return SolveTile<3, 1>::exists(g) ? SolveTile<3, 1>::occupancy(g) : 0;
  return 0;
}

bool solve_launch_narrow(int cg, int g, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                         cudaStream_t st) {
  if (cg == 2) return SolveTile<2, 1>::launch(g, Ds, items, nitems, sms, M, st);
  if (cg == 3) return SolveTile<3, 1>::launch(g, Ds, items, nitems, sms, M, st);
  return false;
}

}  // namespace zr
