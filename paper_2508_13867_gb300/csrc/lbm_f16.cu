// Lattice-Boltzmann kernels instantiated for FP16 (scaled by 2^12) population storage.
#include "lbm_kernels.cuh"

namespace uqlb {

const StorageOps& storage_ops_f16() {
    static const StorageOps ops = make_storage_ops<__half>();
    return ops;
}

}  // namespace uqlb
