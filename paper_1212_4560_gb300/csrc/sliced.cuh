// sliced.cuh -- layout of the digit-sliced operands (Ozaki, Ogita, Oishi &
// Rump, "Error-free transformations of matrix multiplication", Numer.
// Algorithms 2012), shared by the slicing kernels and the tensor-core
// product.
//
// An FP64 operand row (of A) or column (of B) is scaled by a power of two
// 2^e > max |x| and cut into ND signed 7-bit digits:
//   x = 2^e (sum_{t=1..ND} d_t 2^{-7t} + r),   |d_1| <= 128, |d_t| <= 64 (t > 1), |r| <= 2^-(7 ND + 1).
// Each digit is a small integer, exact in BF16.  An operand row holds its ND
// digit slices side by side along K: digit t of entry k at [(t-1) Kpad + k],
// Kpad = K rounded up to the k-tile, padding zero.
//
// The product keeps the digit pairs (t, u) with g = t + u <= ND + 1, summed
// by group:  P_g = sum_{t+u=g} sum_k d_t(a_ik) d_u(b_kj), an integer with
// |P_g| <= (g + 1) 2^12 K, so FP32 accumulation is exact for g <= 7 at
// K <= 512; only the last group g = ND + 1 may round, at 2^-24 of a term
// 2^-7 ND below the leading one.  Then
//   (A B)_ij ~ 2^{e_i + f_j} sum_{g=2..ND+1} 2^{-7g} P_g,
// and the dropped pairs and the truncation leave about 2^-(7 ND - 1) of
// 2^{e_i + f_j} per term of the sum over k.
#pragma once

namespace genp {
namespace sliced {

// Supported digit counts: 3 (about 19 correct bits on Gaussian data), 4
// (about 26), 5 (about 33), 6 (about 40) and 7 (about 47).  ND groups of 64
// TMEM columns each.  The factorization takes 5 to 7 digits; a product that
// only has to be as accurate as the factors it feeds (A G) may take fewer.
__host__ __device__ constexpr bool supported(int nd) { return nd >= 3 && nd <= 7; }
__host__ __device__ constexpr bool factor_supported(int nd) { return nd >= 5 && nd <= 7; }

}  // namespace sliced
}  // namespace genp
