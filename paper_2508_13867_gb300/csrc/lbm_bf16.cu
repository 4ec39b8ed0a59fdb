// Lattice-Boltzmann kernels instantiated for BF16 population storage.
#include "lbm_kernels.cuh"

namespace uqlb {

const StorageOps& storage_ops_bf16() {
    static const StorageOps ops = make_storage_ops<__nv_bfloat16>();
    return ops;
}

}  // namespace uqlb
