// zr_solve_wide.cu -- solve instances with 4, 6 and 8 right-hand sides per
// consumer thread, for the larger S they serve (4 to 8 consumer warps).
#include "zr_solve.cuh"

namespace zr {

int solve_occupancy_wide(int cg, int g) {
  if (cg == 4) return SolveTile<4, 4>::exists(g) ? SolveTile<4, 4>::occupancy(g) : 0;
  if (cg == 6) return SolveTile<6, 4>::exists(g) ? SolveTile<6, 4>::occupancy(g) : 0;
  if (cg == 8) return SolveTile<8, 4>::exists(g) ? SolveTile<8, 4>::occupancy(g) : 0;
  return 0;
}

bool solve_launch_wide(int cg, int g, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                       cudaStream_t st) {
  if (cg == 4) return SolveTile<4, 4>::launch(g, Ds, items, nitems, sms, M, st);
  if (cg == 6) return SolveTile<6, 4>::launch(g, Ds, items, nitems, sms, M, st);
  if (cg == 8) return SolveTile<8, 4>::launch(g, Ds, items, nitems, sms, M, st);
  return false;
}

}  // namespace zr
