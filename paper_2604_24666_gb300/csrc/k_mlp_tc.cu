// k_mlp_tc.cu -- tensor-core (tcgen05 / TMEM) MLP forward, BF16 or FP16
// operands with FP32 accumulation.
#include "nif_internal.cuh"

nif_status nif_mlp_fwd_tc_run(nif_handle* h, const void* x, int dtype, const uint32_t* n_dev, int64_t n_max,
                              float* out, cudaStream_t s) {
    NifProf prof_(h, "mlp_fwd_tc", s);
    (void)x; (void)dtype; (void)n_dev; (void)n_max; (void)out; (void)s;
    return nif_fail(h, NIF_ERR_STATE, "tensor-core MLP not built yet");
}
