// gas.cu -- generalised-active-space (GAS) restrictions of the determinant
// space (Sec. "Generalized Active Space"; the CAAB types of Eqs. 2gas and
// 3gas1-3gas4 enumerate the same kind of subspace occupations).
//
// The orbitals are split into ordered subspaces, subspace j holding the next
// sizes[j] orbitals.  A determinant is kept iff for every j the electrons
// (alpha + beta) in subspaces 0..j number between cmin[j] and cmax[j] (the
// accumulated form of the occupation limits).  The restricted CI problem is
// P H P with P the projector onto the kept determinants.  One lower limit can
// be carried by the context's own addressing: a context built on a level split
// after e orbitals (levels = electrons outside them, at most N - cmin) holds
// exactly the determinants with at least cmin electrons inside (iscsi_init_gas
// picks the most restrictive such limit, setup.cu builds the strings with it).
// The limits the addressing does not carry are a mask, applied here: sigma is
// computed on the context's space and its entries outside the GAS space are
// set to zero, and so are the input's (public sigma calls) or the start
// vectors' (Davidson, propagation); a mask costs what the context's space
// costs plus two streaming passes.
//
// Device data: per string its electron count in each subspace, one byte each,
// packed into a 64-bit word (at most 8 subspaces; at most 16 electrons per
// spin, so the alpha and beta words add without carries); the mask, one byte
// per determinant.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.cuh"

namespace iscsi {

namespace {

struct GasLimits {
  int nspace;
  int edge[kGasMaxSpaces + 1];  // first orbital of each subspace, edge[nspace] = n
  int lo[kGasMaxSpaces], hi[kGasMaxSpaces];
};

// occ[i] = packed electron counts per subspace of string i
__global__ void k_gas_occ(const int16_t* __restrict__ orbs, int count, int ne, GasLimits L,
                          unsigned long long* __restrict__ occ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long w = 0;
    for (int e = 0; e < ne; ++e) {
      const int p = orbs[i * ne + e];
      int j = 0;
      while (j + 1 < L.nspace && p >= L.edge[j + 1]) ++j;
      w += 1ull << (8 * j);
    }
    occ[i] = w;
  }
}

// mask[off[a] + b] for every alpha string a and allowed beta string b: one
// block per alpha string, threads along its beta strings
__global__ void k_gas_mask(const long long* __restrict__ off, int acount, const unsigned long long* __restrict__ occa,
                           const unsigned long long* __restrict__ occb, GasLimits L, uint8_t* __restrict__ mask) {
  for (int a = blockIdx.x; a < acount; a += gridDim.x) {
    const long long base = off[a];
    const int nbeta = (int)(off[a + 1] - base);
    const unsigned long long wa = occa[a];
    for (int b = threadIdx.x; b < nbeta; b += blockDim.x) {
      const unsigned long long w = wa + occb[b];
      int acc = 0;
      bool ok = true;
      for (int j = 0; j < L.nspace; ++j) {
        acc += (int)((w >> (8 * j)) & 0xffu);
        ok = ok && acc >= L.lo[j] && acc <= L.hi[j];
      }
      mask[base + b] = ok ? 1 : 0;
    }
  }
}

// dst[v][e] = mask[e] ? src[v][e] : 0 (src == dst allowed)
__global__ void k_gas_project(const double* src, double* dst, const uint8_t* __restrict__ mask, long long ndet,
                              int nvec) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ndet;
       e += (long long)gridDim.x * blockDim.x) {
    const bool keep = mask[e] != 0;
    for (int v = 0; v < nvec; ++v) {
      const long long i = (long long)v * ndet + e;
      dst[i] = keep ? src[i] : 0.0;
    }
  }
}

}  // namespace

int gas_set(Context& ctx, int nspace, const int* sizes, const int* cmin, const int* cmax) {
  cudaStream_t st = stream();
  if (nspace == 0) {
    ctx.gas_nspace = 0;
    ctx.gas_ndet = ctx.ndet;
    ctx.gas_mask.release();
    ctx.gas_mask_h.clear();
    ctx.gas_in.release();
    return kOk;
  }
  const int N = ctx.na + ctx.nb;
  if (nspace < 1 || nspace > kGasMaxSpaces || !sizes || !cmin || !cmax) {
    set_error("iscsi_set_gas: 1 to 8 subspaces with sizes and limits (or 0 subspaces to remove the restriction)");
    return kErrArg;
  }
  GasLimits L{};
  L.nspace = nspace;
  int acc = 0;
  for (int j = 0; j < nspace; ++j) {
    if (sizes[j] < 1 || cmin[j] < 0 || cmax[j] < cmin[j] || cmax[j] > N) {
      set_error("iscsi_set_gas: subspace sizes >= 1 and limits 0 <= cmin <= cmax <= electrons");
      return kErrArg;
    }
    L.edge[j] = acc;
    acc += sizes[j];
    L.lo[j] = cmin[j];
    L.hi[j] = cmax[j];
  }
  L.edge[nspace] = acc;
  if (acc != ctx.n) {
    set_error("iscsi_set_gas: subspace sizes must add up to the orbital count");
    return kErrArg;
  }
  // unrestricted until the new mask is complete (a failure below leaves no restriction)
  ctx.gas_nspace = 0;
  ctx.gas_ndet = ctx.ndet;
  DevBuf occ[2];
  for (int s = 0; s < 2; ++s) {
    const SpinSpace& S = ctx.sp[s];
    ISCSI_TRY(occ[s].alloc(sizeof(unsigned long long) * S.count));
    k_gas_occ<<<std::min(launch_blocks(S.count, 256), 4096), 256, 0, st>>>(S.orbs.as<int16_t>(), S.count, S.ne, L,
                                                                          occ[s].as<unsigned long long>());
    ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
  }
  ISCSI_TRY(ctx.gas_mask.alloc(ctx.ndet));
  const int acount = ctx.sp[0].count;
  k_gas_mask<<<std::min(acount, 152 * 64), 256, 0, st>>>(ctx.off.as<long long>(), acount,
                                                         occ[0].as<unsigned long long>(),
                                                         occ[1].as<unsigned long long>(), L,
                                                         ctx.gas_mask.as<uint8_t>());
  ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  ctx.gas_mask_h.resize(ctx.ndet);
  ISCSI_CUDA(cudaMemcpyAsync(ctx.gas_mask_h.data(), ctx.gas_mask.p, ctx.ndet, cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  long long kept = 0;
  for (uint8_t m : ctx.gas_mask_h) kept += m;
  ctx.gas_nspace = nspace;
  ctx.gas_ndet = kept;
  return kOk;
}

int gas_project(const Context& ctx, const double* src, double* dst, int nvec, cudaStream_t st) {
  if (ctx.gas_nspace == 0) {
    if (src != dst)
      ISCSI_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * ctx.ndet * nvec, cudaMemcpyDeviceToDevice, st));
    return kOk;
  }
  k_gas_project<<<std::min(launch_blocks(ctx.ndet, 256), 152 * 16), 256, 0, st>>>(
      src, dst, ctx.gas_mask.as<uint8_t>(), ctx.ndet, nvec);
  ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

}  // namespace iscsi
