// Layered-texture synthesis variant (Sec. 4.2): placeholder.
#include <cuda_runtime.h>

#include "internal.h"

namespace scwp {

cudaError_t launch_layered(PatchDev&, const SynthParams&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace scwp
