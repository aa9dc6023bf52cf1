// Host-side access to a context's own stepping from padded FP64 states
// [2][12][plane] (both grids, interior valid), for the adjoint's forward
// sweeps.  Defined in fdcgks_api.cu.
#pragma once

#include "../../include/fdcgks.h"

namespace fdk {
// load a padded FP64 state into the context (split into float-float pairs on
// the mixed path); marks the state loaded, does not validate it
fdcgks_status ctx_load_padded(fdcgks_t c, const double* in);
// one step of the context's precision from `in` to `out` (both padded FP64);
// the context's state is overwritten, its time is kept
fdcgks_status ctx_replay_step(fdcgks_t c, double dt, const double* in, double* out);
}  // namespace fdk
