// smc_mlp.h -- the surrogate network: IN -> 128 -> 128 -> 128 -> 1 (ReLU
// hidden layers, logistic output), BF16 weights and activations with FP32
// accumulation on the tensor cores, FP32 master weights and Adam.
#pragma once
#include <stdint.h>

#define MLP_IN 16    // input features, zero-padded
#define MLP_H 128    // hidden width

// Flat FP32 parameter vector: W1 [H][IN], b1 [H], W2 [H][H], b2 [H], W3 [H][H],
// b3 [H], w4 [H], b4 [1].
enum {
    MLP_OFF_W1 = 0,
    MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN,
    MLP_OFF_W2 = MLP_OFF_B1 + MLP_H,
    MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H,
    MLP_OFF_W3 = MLP_OFF_B2 + MLP_H,
    MLP_OFF_B3 = MLP_OFF_W3 + MLP_H * MLP_H,
    MLP_OFF_W4 = MLP_OFF_B3 + MLP_H,
    MLP_OFF_B4 = MLP_OFF_W4 + MLP_H,
    MLP_NPARAM = MLP_OFF_B4 + 1
};

struct smc_mlp;
// The network's number of input features (library-internal).
int smc_mlp_inputs(const smc_mlp *m);
