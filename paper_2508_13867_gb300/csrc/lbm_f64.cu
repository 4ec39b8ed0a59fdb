// Lattice-Boltzmann kernels instantiated for FP64 population storage.
#include "lbm_kernels.cuh"

namespace uqlb {

const StorageOps& storage_ops_f64() {
    static const StorageOps ops = make_storage_ops<double>();
    return ops;
}

}  // namespace uqlb
