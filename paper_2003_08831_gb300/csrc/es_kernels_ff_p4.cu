// Float-float (ES_FP64X) kernel instantiations for LGL degree p = 3 (P1 = 4 points per direction).
#include "es_kernels.cuh"

namespace es {
template struct Launcher<4, ff>;
}  // namespace es
