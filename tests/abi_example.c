/*
 * A plain C99 caller of the library (compiled and run by test_abi_host.py):
 * the header must compile as C, the host-only sweep planner must work
 * without a GPU, and state creation must either succeed (a GPU is present:
 * H on every qubit of |0..0> is QFT|0>, fidelity 1) or fail cleanly with
 * QSIM_ERR_CUDA and a message.
 */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "qsim.h"

#define NQ 10

static void hadamard(double *m)
{
    const double r = 1.0 / sqrt(2.0);
    memset(m, 0, 32 * sizeof(double));
    m[0] = r;
    m[2] = r;
    m[4] = r;
    m[6] = -r;
}

int main(void)
{
    int ntargets[NQ], targets[2 * NQ], lo[NQ], h[NQ], H[4 * NQ];
    double matrices[32 * NQ];
    int q, ns;
    qsim_t st = NULL;
    qsim_status s;
    qsim_ref ref;
    double F = 0.0;

    for (q = 0; q < NQ; ++q) {
        ntargets[q] = 1;
        targets[2 * q] = q;
        targets[2 * q + 1] = 0;
        hadamard(matrices + 32 * q);
    }
    ns = qsim_plan_sweeps(NQ, 4, 2, 512, NQ, ntargets, targets, matrices, lo, h, H, NQ);
    if (ns < 1) {
        printf("plan failed %d\n", ns);
        return 1;
    }
    printf("sweeps %d\n", ns);

    s = qsim_create(&st, NQ, 8, QSIM_CODEC_REL, 1e-4);
    if (s != QSIM_OK) {
        printf("create %d %s\n", (int)s, qsim_last_error(NULL));
        return s == QSIM_ERR_CUDA ? 0 : 1;
    }
    for (q = 0; q < NQ; ++q) {
        s = qsim_apply_gate(st, matrices + 32 * q, &q, 1, NULL, 0, ~0ULL);
        if (s != QSIM_OK) {
            printf("apply %d %s\n", (int)s, qsim_last_error(st));
            return 1;
        }
    }
    memset(&ref, 0, sizeof ref);
    ref.kind = QSIM_REF_QFT_BASIS;
    ref.x = 0;
    s = qsim_fidelity(st, &ref, &F, NULL);
    qsim_destroy(st);
    if (s != QSIM_OK || !(F > 0.9999)) {
        printf("fidelity %d %.12f\n", (int)s, F);
        return 1;
    }
    printf("fidelity %.12f\n", F);
    return 0;
}
