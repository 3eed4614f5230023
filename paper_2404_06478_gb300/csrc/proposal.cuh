// proposal.cuh — constants and buffer layouts of the learned proposal (the
// set encoder beside the paper's candidate scan; see proposal.cu).
#pragma once

#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

namespace laue {
namespace lp {

constexpr int KSET = 128;   // spots per set: the seed + 127 neighbours (a multiple of 128)
constexpr int NF = 64;      // feature width (14 used)
constexpr int WIDTH = 256;  // per-spot MLP width
constexpr int HEADW = 256;  // head hidden width
constexpr int NHYP = 8;     // hypotheses per set
constexpr int NOUT = 9 * NHYP;
constexpr int NOUTP = 128;  // NOUT padded to a tensor-core tile (zero rows / columns beyond NOUT)
constexpr float XSCALE = 2.5f;
constexpr float LAMBDA_X = 0.1f;
constexpr float BETA = 0.05f;
constexpr float DSCALE = 200.0f;
constexpr float HALFS = 128.0f;
constexpr int kMaxSplits = 64;   // split-K partials of the weight gradients

// FP32 parameter vector: W1 (256 x 64), b1, W2 (256 x 256), b2, W3, b3,
// W4 (256 x 512), b4, W5 (72 x 256), b5; weights row-major [out][in].
constexpr size_t oW1 = 0;
constexpr size_t ob1 = oW1 + (size_t)WIDTH * NF;
constexpr size_t oW2 = ob1 + WIDTH;
constexpr size_t ob2 = oW2 + (size_t)WIDTH * WIDTH;
constexpr size_t oW3 = ob2 + WIDTH;
constexpr size_t ob3 = oW3 + (size_t)WIDTH * WIDTH;
constexpr size_t oW4 = ob3 + WIDTH;
constexpr size_t ob4 = oW4 + (size_t)HEADW * 2 * WIDTH;
constexpr size_t oW5 = ob4 + HEADW;
constexpr size_t ob5 = oW5 + (size_t)NOUT * HEADW;
constexpr size_t kParams = ob5 + NOUT;

inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Network buffer (bytes): FP32 params, Adam moments m and v, gradients,
// BF16 copies of the weights (the per-spot ones row-major and transposed,
// W4 row-major, W5 row-major padded to NOUTP rows), split-K partials, the
// Adam step counter.
struct NetLayout {
    size_t params, adam_m, adam_v, grads, W1h, W2h, W3h, W2t, W3t, W4h, W5h, partial, step, total;
};
inline NetLayout net_layout() {
    NetLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = al256(o + bytes); return r; };
    L.params = take(kParams * 4);
    L.adam_m = take(kParams * 4);
    L.adam_v = take(kParams * 4);
    L.grads = take(kParams * 4);
    L.W1h = take((size_t)WIDTH * NF * 2);
    L.W2h = take((size_t)WIDTH * WIDTH * 2);
    L.W3h = take((size_t)WIDTH * WIDTH * 2);
    L.W2t = take((size_t)WIDTH * WIDTH * 2);
    L.W3t = take((size_t)WIDTH * WIDTH * 2);
    L.W4h = take((size_t)HEADW * 2 * WIDTH * 2);
    L.W5h = take((size_t)NOUTP * HEADW * 2);
    L.partial = take((size_t)kMaxSplits * WIDTH * WIDTH * 4);
    L.step = take(256);
    L.total = o;
    return L;
}

// Batch buffer (bytes) for B sets of KSET spots (Ms = B KSET rows).  The
// head's tensor-core operands have Bp = B rounded up to 128 rows; the rows
// beyond B hold zero features and zero errors.
struct BatchLayout {
    size_t X, H1, H2, H3, dZ3, dZ2, dZ1;  // BF16 per-spot arrays, row-major [spots][channels]
    size_t F, nvalid, Rt, xt, svalid, pool, amax, O, dO, loss, dbest, hbest, inv_nval;
    size_t poolh, H4h, dZ4h, dOh;  // BF16 head operands [Bp][512], [Bp][256], [Bp][256], [Bp][NOUTP]
    size_t Opad, dPool;            // FP32 [Bp][NOUTP], [Bp][512]
    size_t total;
    long long Ms;
    int Bp;
};
inline BatchLayout batch_layout(int B) {
    BatchLayout L;
    size_t o = 0;
    long long Ms = (long long)B * KSET;
    L.Ms = Ms;
    auto take = [&](size_t bytes) { size_t r = o; o = al256(o + bytes); return r; };
    L.X = take((size_t)Ms * NF * 2);
    L.H1 = take((size_t)Ms * WIDTH * 2);
    L.H2 = take((size_t)Ms * WIDTH * 2);
    L.H3 = take((size_t)Ms * WIDTH * 2);
    L.dZ3 = take((size_t)Ms * WIDTH * 2);
    L.dZ2 = take((size_t)Ms * WIDTH * 2);
    L.dZ1 = take((size_t)Ms * WIDTH * 2);
    L.F = take((size_t)B * 9 * 4);
    L.nvalid = take((size_t)B * 4);
    L.Rt = take((size_t)B * 9 * 4);
    L.xt = take((size_t)B * 3 * 4);
    L.svalid = take((size_t)B * 4);
    L.pool = take((size_t)B * 2 * WIDTH * 4);
    L.amax = take((size_t)B * WIDTH * 4);
    L.O = take((size_t)B * NOUT * 4);
    L.dO = take((size_t)B * NOUT * 4);
    L.loss = take((size_t)B * 4);
    L.dbest = take((size_t)B * 4);
    L.hbest = take((size_t)B * 4);
    L.inv_nval = take(256);
    const int Bp = (B + 127) / 128 * 128;
    L.Bp = Bp;
    L.poolh = take((size_t)Bp * 2 * WIDTH * 2);
    L.H4h = take((size_t)Bp * HEADW * 2);
    L.dZ4h = take((size_t)Bp * HEADW * 2);
    L.dOh = take((size_t)Bp * NOUTP * 2);
    L.Opad = take((size_t)Bp * NOUTP * 4);
    L.dPool = take((size_t)Bp * 2 * WIDTH * 4);
    L.total = o;
    return L;
}

}  // namespace lp
}  // namespace laue
