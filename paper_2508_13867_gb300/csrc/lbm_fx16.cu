// Lattice-Boltzmann kernels instantiated for 16-bit fixed-point population storage (per-sample
// quanta of the rest, axis and diagonal populations).
#include "lbm_kernels.cuh"

namespace uqlb {

const StorageOps& storage_ops_fx16() {
    static const StorageOps ops = make_storage_ops<int16_t>();
    return ops;
}

}  // namespace uqlb
