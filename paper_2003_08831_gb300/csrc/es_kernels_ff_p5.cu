// Float-float (ES_FP64X) kernel instantiations for LGL degree p = 4 (P1 = 5 points per direction).
#include "es_kernels.cuh"

namespace es {
template struct Launcher<5, ff>;
}  // namespace es
