// BF16 tensor-core Rayleigh-Ritz products (tcgen05 path): not built yet.
#include "hub_internal.cuh"

namespace hub {

int launch_gram_bf16(hub_t h, const void*, int, const void*, int, int, int, double, bool, double*) {
    return fail(h, HUB_EINVAL, "HUB_MIXED_BF16 products are not available in this build");
}

int launch_rotate_bf16(hub_t h, const void*, int, const double*, int, int, void*, int) {
    return fail(h, HUB_EINVAL, "HUB_MIXED_BF16 products are not available in this build");
}

}  // namespace hub
