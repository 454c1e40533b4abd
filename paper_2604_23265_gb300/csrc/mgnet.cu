// MgNet preconditioner (Sec. 3).
#include "mgnet_internal.h"

namespace rte {

void mgnet_prepare(mgnet*, rte_ctx*) {
    throw StatusError{RTE_ENOTSUP, "MgNet preconditioner not built"};
}

void mgnet_precondition(mgnet*, rte_ctx*, const double*, float*) {
    throw StatusError{RTE_ENOTSUP, "MgNet preconditioner not built"};
}

}  // namespace rte
