// Arguments of the regrid kernel (mg_regrid.cu), shared with the host
// (mg_capi.cu).
#pragma once
#include "mg_plan.h"

namespace mgk {

// The array `buf` (complex, the launching context's precision) holds a state
// on the grid centred at (src_ctrl[0..D), src_ctrl[8..8+D)), a device control
// block.  One launch carries it onto the grid centred at (qt, pt), or at
// (qt, source p) with keep_p.  With commit, the launching context's own
// centres become (qt, pt).
struct RegridArgs {
  double qt[MAXD], pt[MAXD];
  const double* src_ctrl;
  void* buf;
  int keep_p, commit;
};

}  // namespace mgk
