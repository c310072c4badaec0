// Matrix-free operator (tensor-core logits); filled in by the tcgen05 kernels.
#include "laker_device.cuh"

laker_status mf_matvec_launch(laker_ctx* ctx, const laker_op* op, const double* pin, const double* z, double* pout,
                              double* w, PcgScalars* sc, double* partials, int fuse, float* pbuf, float* wbuf) {
    (void)op; (void)pin; (void)z; (void)pout; (void)w; (void)sc; (void)partials; (void)fuse; (void)pbuf; (void)wbuf;
    return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator not built");
}
