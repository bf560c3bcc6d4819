// Tensor-core (tcgen05) linewidth path: placeholder until the kernels land.
#include "common.h"

phx_status phx_gamma_tc(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                        const double* nB, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                        int prec, double* gacc, double* wacc, cudaStream_t s) {
    (void)f; (void)freq; (void)evec; (void)nB; (void)irr_host; (void)n_irr; (void)gp; (void)prec;
    (void)gacc; (void)wacc; (void)s;
    return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core precision not built yet");
}
