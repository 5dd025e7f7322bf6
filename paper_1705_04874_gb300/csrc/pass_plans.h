// The FFT plans of the derivative passes, one X(n, R1, R2, R3) per candidate:
// radices of the stages in order, R3 = 1 for a two-stage plan.  The first
// candidate of a length is the default; es_model_autotune may pick another.
// Through the C ABI a plan is named (R1, n / R1).  Every radix has a register
// DFT in fft_pass.cuh (2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 25).
#pragma once

#define ES_PLANS(X)                                                                                  \
    X(16, 4, 4, 1)                                                                                   \
    X(32, 8, 4, 1) X(32, 4, 8, 1)                                                                    \
    X(48, 12, 4, 1) X(48, 4, 12, 1)                                                                  \
    X(64, 16, 4, 1) X(64, 8, 8, 1) X(64, 4, 16, 1)                                                   \
    X(75, 5, 15, 1) X(75, 3, 5, 5) X(75, 15, 5, 1)                                                   \
    X(80, 16, 5, 1) X(80, 5, 16, 1)                                                                  \
    X(96, 16, 6, 1) X(96, 6, 16, 1)                                                                  \
    X(125, 5, 5, 5) X(125, 25, 5, 1)                                                                 \
    X(128, 16, 8, 1) X(128, 8, 16, 1)                                                                \
    X(160, 16, 10, 1) X(160, 10, 16, 1)                                                              \
    X(192, 16, 12, 1) X(192, 12, 16, 1)                                                              \
    X(256, 16, 16, 1)
