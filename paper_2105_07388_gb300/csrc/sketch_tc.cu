// Right sketch on the 5th-generation tensor cores (BF16x3 split of A).
#include "internal.h"

namespace re {

bool tc_supported(const MatView&) { return false; }

cudaError_t launch_right_tc(const MatView&, const uint16_t*, int64_t, int, float*, int64_t, int*,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace re
