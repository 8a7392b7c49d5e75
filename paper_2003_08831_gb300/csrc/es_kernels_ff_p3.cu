// Float-float (ES_FP64X) kernel instantiations for LGL degree p = 2 (P1 = 3 points per direction).
#include "es_kernels.cuh"

namespace es {
template struct Launcher<3, ff>;
}  // namespace es
