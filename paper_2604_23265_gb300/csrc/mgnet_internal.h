// Internal interface between the solver and the MgNet preconditioner.
#pragma once

#include "rte_internal.h"

namespace rte {

// Computes (once per medium and weight version) what the network needs for
// this context: the CoeffNet features a^[l], a^{-1,[l]} of the medium.
void mgnet_prepare(mgnet* net, rte_ctx* ctx);

// z = D Net(v): the learned preconditioner applied to one Krylov vector.
void mgnet_precondition(mgnet* net, rte_ctx* ctx, const double* v, float* z);

// The same for B vectors of B contexts of one grid size (a lockstep group):
// the tensor-core layers run once for all of them (batches of up to 16), each
// sample with its own medium; every z_b is the same bits as alone.
void mgnet_precondition_batch(mgnet* net, rte_ctx* const* ctxs, const double* const* v, float* const* z, int B);

// The same two for an FP32 input vector (the hi plane of a df64 Krylov
// vector): the tensor-core forward reads it directly (its convolutions round
// the input to BF16 and its projection adds it in FP32, so the FP32 input
// changes nothing); the CUDA-core forward widens it to FP64 first.
void mgnet_precondition_f(mgnet* net, rte_ctx* ctx, const float* v, float* z);
void mgnet_precondition_batch_f(mgnet* net, rte_ctx* const* ctxs, const float* const* v, float* const* z, int B);

}  // namespace rte
