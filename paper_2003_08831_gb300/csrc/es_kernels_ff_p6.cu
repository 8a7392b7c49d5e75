// Float-float (ES_FP64X) kernel instantiations for LGL degree p = 5 (P1 = 6 points per direction).
#include "es_kernels.cuh"

namespace es {
template struct Launcher<6, ff>;
}  // namespace es
