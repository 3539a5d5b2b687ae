/* A plain C caller of the library's C ABI (no Python): a batch of mode-sum instances, evolved to
 * t = 0.5 with the spectrum and the TTF quantities tracked every 0.25, then the fields of one
 * instance read back.  Prints one line per instance: status, mass, E, N, T at the last snapshot;
 * then the checksum of instance 0's Pi.  Used by tests/test_gpu_c_consumer.py. */
#include <stdio.h>
#include <stdlib.h>

#include "adscl.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        adscl_status st_ = (call);                                                    \
        if (st_ != ADSCL_OK) {                                                        \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, (int)st_,                  \
                    ctx ? adscl_last_error(ctx) : "");                                \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

int main(void)
{
    enum { B = 3, K = 6, J = 16, S = 3 };
    const int32_t N[B] = {257, 513, 1025};
    adscl_config cfg = {0};
    cfg.num_instances = B;
    cfg.N = N;
    cfg.cfl = 0.5;
    cfg.ko_sigma = 0.5;
    cfg.collapse_threshold = 1.0 / 128.0;
    cfg.out_dt = 0.25;
    adscl_ctx *ctx = NULL;
    CHECK(adscl_create(&cfg, &ctx));
    double a[B * K];
    for (int b = 0; b < B; ++b)
        for (int k = 0; k < K; ++k) a[b * K + k] = 0.1 * (b + 1) / (1.0 + k * k);
    CHECK(adscl_set_initial_modes(ctx, a, K, 0));
    double t_hist[S * B], ttf_hist[S * B * 3];
    CHECK(adscl_track(ctx, 0.0, 0.25, S, J, ADSCL_PREC_FP64, t_hist, ttf_hist, NULL, 0));
    double tr[B], tc[B], mass[B];
    int32_t status[B];
    CHECK(adscl_evolve(ctx, 0.5, tr, tc, mass, status, 0));
    for (int b = 0; b < B; ++b) {
        const double *q = ttf_hist + ((S - 1) * B + b) * 3;
        printf("%d %d %.17g %.17g %.17g %.17g %.17g\n", b, (int)status[b], tr[b], mass[b], q[0], q[1], q[2]);
    }
    double *Pi = (double *)malloc(sizeof(double) * N[0]);
    CHECK(adscl_get_state(ctx, 0, NULL, Pi, NULL, NULL, 0));
    double sum = 0.0;
    for (int i = 0; i < N[0]; ++i) sum += Pi[i] * (i + 1);
    printf("checksum %.17g\n", sum);
    free(Pi);
    adscl_destroy(ctx);
    return 0;
}
