// Host side of the TMA tensor maps: the driver's cuTensorMapEncodeTiled,
// looked up once through the runtime (no link dependency on libcuda).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

namespace spp {

// nullptr if the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace spp
