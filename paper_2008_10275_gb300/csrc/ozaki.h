// FP64 Gram products G = A^T B of tall factors on the BF16 tensor cores by
// an error-free splitting (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every column of A and B is scaled by a power of two fixed by its largest
// entry and written as a 56-bit fixed-point integer, cut into 8 balanced
// base-128 digits (the slices: the first in [-128, 128], the others in
// [-64, 63]); a digit is exact in BF16.  The product of two slices summed over
// at most 256 rows stays below 2^24, so the FP32 accumulation of the tensor
// core is exact there; the slice products are grouped by level t + u (8
// levels, pairs with t + u >= 8 dropped: below 2^-54 of the column scales),
// read out of tensor memory every 256 rows and summed as integers.  The only
// rounding is the 56-bit fixed point of each input and the final FP64
// combination of the 8 levels: the result is as accurate as an FP64 Gram.
#pragma once

#include "dense.h"

namespace lrfsi {

// Workspace (bytes) of ozaki_gram for nbatch products of M rows with at most
// pmax columns of A and qmax of B (B == A needs no slices of its own).
size_t ozaki_work_bytes(int nbatch, long M, int pmax, int qmax);
// G_b = A_b^T B_b for the descriptors (GramDesc, gates honoured); work: at
// least ozaki_work_bytes(...) bytes, 256-byte aligned.
int ozaki_gram(const GramDesc* d, int nbatch, long M, void* work, size_t work_bytes, cudaStream_t s);

// flag = 1 if a pipeline wait of the tensor-core Gram ran out since the last
// call (the products of that launch are wrong); synchronises the stream.
int ozaki_error(cudaStream_t s, int* flag);

// Tall GEMMs on the tensor cores (GemmDesc::tc, m >= 2048, 1 <= k <= 400).
bool ozaki_gemm_eligible(const GemmDesc<double>& g);
size_t ozaki_gemm_work_bytes(const GemmDesc<double>* d, int n);
int ozaki_gemm(const GemmDesc<double>* d, int n, void* work, size_t work_bytes, cudaStream_t s);

// Gram product path: 1 = tensor cores (this file), 0 = FP64 SIMT kernels.
int gram_path();
void set_gram_path(int p);

}  // namespace lrfsi
