// Lattice-Boltzmann kernels instantiated for FP32 population storage.
#include "lbm_kernels.cuh"

namespace uqlb {

const StorageOps& storage_ops_f32() {
    static const StorageOps ops = make_storage_ops<float>();
    return ops;
}

}  // namespace uqlb
