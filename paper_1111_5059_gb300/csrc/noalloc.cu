// dwf_apply_Mpc_noalloc: the even-odd Schur operator without any device
// memory allocation during the call.
//
// dwf_apply_Mpc takes its packed FP64 fields from the handle's workspace,
// which the library allocates with cudaMalloc on first use (and its
// fifth-dimension coefficient tables with cudaMalloc on the first call with
// a new mass).  Code that must not allocate while it runs -- code under an
// allocator that owns all device memory, or a loop that may not stall on the
// driver -- calls this entry point instead.  Its scratch is one file-scope
// device array of fixed size, present on every GPU that loads the library
// until the process exits; the fifth-dimension operators are passed to the
// kernels as by-value coefficients, so no table is allocated either.
#include <cmath>
#include <mutex>

#include "dwf_internal.h"

namespace dwf {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[DWF_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is not a device address).
dwf_status scratch_address(dwf_lattice* L, void** out) {
  int dev = 0;
  DWF_CUDA(L, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    DWF_CUDA(L, cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return DWF_OK;
}

}  // namespace

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_apply_Mpc_noalloc(dwf_lattice_t L, double m, int dag, const void* in, void* out) {
  if (!L || !in || !out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_noalloc: null argument");
  if (in == out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_noalloc: in and out must not alias");
  if (!std::isfinite(m)) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_noalloc: non-finite mass");
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "gauge field not set");
  const size_t fb = (field_bytes(L, DWF_F64) + 255) / 256 * 256;
  if (4 * fb > (size_t)DWF_NOALLOC_SCRATCH_BYTES)
    return fail(L, DWF_ERR_INVALID_ARG,
                "dwf_apply_Mpc_noalloc: lattice too large for the fixed scratch (needs " + std::to_string(4 * fb) +
                    " bytes, DWF_NOALLOC_SCRATCH_BYTES = " + std::to_string((size_t)DWF_NOALLOC_SCRATCH_BYTES) + ")");
  SOps ops{};
  ops.m = m;
  fifth_descriptors(L->p, L->Ls, m, ops.desc);
  for (int k = 0; k < SOps::NKIND; ++k)
    if (ops.desc[k].kind == 2)
      return fail(L, DWF_ERR_INVALID_ARG,
                  "dwf_apply_Mpc_noalloc: these Moebius parameters need the dense fifth-dimension fallback");
  void* base = nullptr;
  DWF_TRY(scratch_address(L, &base));
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  ops.d64 = reinterpret_cast<double*>(base);  // never dereferenced: every descriptor is structured
  ops.d32 = reinterpret_cast<float*>(base);
  Field xe, ye, t, u;
  xe.v = p;
  ye.v = p + fb;
  t.v = p + 2 * fb;
  u.v = p + 3 * fb;
  // every word the kernels read is written earlier in this call, so nothing
  // needs clearing: the FP64 per-slice kernels (pack, s-local, hop) read and
  // write only the slices s < Ls, never the padding slot of an odd Ls.  Kernel
  // timing (event creation) is suspended for the call.
  const bool timing = L->timing;
  L->timing = false;
  dwf_status st = launch_pack(L, in, 0, xe);
  HopCall c1, c2;
  c1.ops = c2.ops = &ops;
  if (!dag) {
    // M_pc x = A x - 1/4 Dhop (B A^-1) Dhop (B x)
    if (st == DWF_OK) st = launch_sop(L, xe, t, &ops, SOps::B, 1.0, nullptr, 0.0);
    c1.out_parity = 1;
    c1.in = t;
    c1.out = u;
    c1.eout = SOps::E1;
    c2.out_parity = 0;
    c2.in = u;
    c2.out = ye;
    c2.x = xe;
    c2.has_x = true;
    c2.ex = SOps::A;
    c2.scale = -0.25;
  } else {
    // M_pc^+ x = B^+ (E0^+ x - 1/4 Dhop^+ (E1^+ Dhop^+ x))
    c1.out_parity = 1;
    c1.dag = 1;
    c1.in = xe;
    c1.out = u;
    c1.eout = SOps::E1T;
    c2.out_parity = 0;
    c2.dag = 1;
    c2.in = u;
    c2.out = ye;
    c2.x = xe;
    c2.has_x = true;
    c2.ex = SOps::E0T;
    c2.eout = SOps::BT;
    c2.scale = -0.25;
  }
  if (st == DWF_OK) st = launch_hop(L, c1);
  if (st == DWF_OK) st = launch_hop(L, c2);
  if (st == DWF_OK) st = launch_unpack(L, ye, 0, out, true);
  L->timing = timing;
  if (st != DWF_OK) return st;
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}
