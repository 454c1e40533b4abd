// Internal interface between the solver and the MgNet preconditioner.
#pragma once

#include "rte_internal.h"

namespace rte {

// Computes (once per medium and weight version) what the network needs for
// this context: the CoeffNet features a^[l], a^{-1,[l]} of the medium.
void mgnet_prepare(mgnet* net, rte_ctx* ctx);

// z = D Net(v): the learned preconditioner applied to one Krylov vector.
void mgnet_precondition(mgnet* net, rte_ctx* ctx, const double* v, float* z);

}  // namespace rte
