// Lattice handle, geometry, fifth-dimension operators, packing and the
// operator entry points of the C ABI.
#include <cmath>
#include <cstring>
#include <mutex>

#include "dwf_internal.h"
#include "geometry.h"

static std::mutex g_err_mu;
static std::string g_err;  // last error of calls without a valid handle

namespace dwf {

dwf_status fail(dwf_lattice* L, dwf_status st, const std::string& msg) {
  if (L) {
    L->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = msg;
  }
  return st;
}

dwf_status cuda_check(dwf_lattice* L, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(L, e == cudaErrorMemoryAllocation ? DWF_ERR_OOM : DWF_ERR_CUDA, msg);
}

long field_elems(const dwf_lattice* L) { return L->Vh * 12 * L->Lh * 4; }

size_t field_bytes(const dwf_lattice* L, dwf_prec prec) {
  return (size_t)field_elems(L) * (prec == DWF_F64 ? 8 : prec == DWF_F32 ? 4 : 2);
}

dwf_status check_dev_err(dwf_lattice* L) {
  // the last pinned scalar slot receives the flag
  int* h = reinterpret_cast<int*>(L->hscal + kScalars - 1);
  *h = 0;
  DWF_CUDA(L, cudaMemcpyAsync(h, L->dev_err, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  if (*h != 0) {
    DWF_CUDA(L, cudaMemsetAsync(L->dev_err, 0, sizeof(int), L->stream));
    DWF_CUDA(L, cudaStreamSynchronize(L->stream));
    return fail(L, DWF_ERR_TIMEOUT, "a bounded device wait gave up (asynchronous copy did not complete)");
  }
  return DWF_OK;
}

dwf_status ws_get(dwf_lattice* L, const std::string& name, size_t bytes, void** out) {
  auto it = L->ws.find(name);
  if (it != L->ws.end() && it->second.bytes >= bytes) {
    *out = it->second.p;
    return DWF_OK;
  }
  if (it != L->ws.end()) {
    cudaFree(it->second.p);
    L->ws.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_check(L, e, ("workspace " + name).c_str());
  // zero-filled once: padding slots of odd-Ls fields must read as zero
  e = cudaMemsetAsync(p, 0, bytes, L->stream);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_check(L, e, ("workspace clear " + name).c_str());
  }
  L->ws[name] = Buffer{p, bytes};
  *out = p;
  return DWF_OK;
}

dwf_status field_alloc(dwf_lattice* L, const std::string& name, dwf_prec prec, Field* f) {
  f->prec = prec;
  f->norm = nullptr;
  DWF_TRY(ws_get(L, name, field_bytes(L, prec), &f->v));
  if (prec == DWF_F16) {
    void* n = nullptr;
    DWF_TRY(ws_get(L, name + ".norm", (size_t)L->Vh * L->Lh * 2 * sizeof(float), &n));
    f->norm = reinterpret_cast<float*>(n);
  }
  return DWF_OK;
}

// ---------------------------------------------------------------- fifth dimension (host)

namespace {
typedef std::vector<double> Mat;  // Ls x Ls row-major

Mat eye(int n) {
  Mat a(n * n, 0.0);
  for (int i = 0; i < n; ++i) a[i * n + i] = 1.0;
  return a;
}
Mat lin(double x, const Mat& a, double y, const Mat& b) {
  Mat r(a.size());
  for (size_t i = 0; i < a.size(); ++i) r[i] = x * a[i] + y * b[i];
  return r;
}
Mat mul(const Mat& a, const Mat& b, int n) {
  Mat r(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j) r[i * n + j] += a[i * n + k] * b[k * n + j];
  return r;
}
Mat transpose(const Mat& a, int n) {
  Mat r(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) r[j * n + i] = a[i * n + j];
  return r;
}
bool inverse(const Mat& a, int n, Mat* out) {  // Gauss-Jordan, partial pivoting
  Mat m = a, r = eye(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(m[i * n + c]) > std::fabs(m[p * n + c])) p = i;
    if (std::fabs(m[p * n + c]) < 1e-300) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(m[p * n + j], m[c * n + j]);
        std::swap(r[p * n + j], r[c * n + j]);
      }
    const double inv = 1.0 / m[c * n + c];
    for (int j = 0; j < n; ++j) {
      m[c * n + j] *= inv;
      r[c * n + j] *= inv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = m[i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        m[i * n + j] -= f * m[c * n + j];
        r[i * n + j] -= f * r[c * n + j];
      }
    }
  }
  *out = r;
  return true;
}
// Fifth-dimension hop matrices with the m wall: up: s <- s+1, dn: s <- s-1.
void shifts(int Ls, double m, Mat* up, Mat* dn) {
  *up = Mat(Ls * Ls, 0.0);
  *dn = Mat(Ls * Ls, 0.0);
  for (int s = 0; s < Ls; ++s) {
    if (s + 1 < Ls)
      (*up)[s * Ls + s + 1] += 1.0;
    else
      (*up)[s * Ls + 0] += -m;
    if (s >= 1)
      (*dn)[s * Ls + s - 1] += 1.0;
    else
      (*dn)[s * Ls + Ls - 1] += -m;
  }
}
}  // namespace

void fifth_descriptors(const dwf_params& p, int Ls, double m, SOpDesc* desc) {
  // y = (g1 + d1 Q)(g2 + d2 Q)^-1 x with A = alpha + beta Q, B = b + c Q,
  // alpha = (4-M5) b + 1, beta = (4-M5) c - 1.
  const double b = p.b, c = p.c, w = 4.0 - p.M5;
  const double al = w * b + 1.0, be = w * c - 1.0;
  const double f[SOps::NKIND][4] = {
      {al, be, 1, 0}, {al, be, 1, 0},  // A, AT
      {1, 0, al, be}, {1, 0, al, be},  // AINV, AINVT
      {b, c, 1, 0},   {b, c, 1, 0},    // B, BT
      {1, 0, b, c},   {1, 0, b, c},    // BINV, BINVT
      {b, c, al, be}, {b, c, al, be},  // E1 = B A^-1, E1T
      {al, be, b, c}, {al, be, b, c},  // E0 = A B^-1, E0T
  };
  for (int k = 0; k < SOps::NKIND; ++k) {
    SOpDesc& d = desc[k];
    const double g1 = f[k][0], d1 = f[k][1], g2 = f[k][2], d2 = f[k][3];
    d.trans = k & 1;
    d.dense_kind = k;
    d.g1 = g1;
    d.d1 = d1;
    d.m = m;
    d.has_inv = d2 != 0.0;
    d.ginv = 1.0 / g2;
    d.rho = -d2 / g2;
    const double den = 1.0 + m * std::pow(d.rho, Ls);
    d.c0 = 1.0 / (g2 * den);
    const bool identity = g1 == 1.0 && d1 == 0.0 && g2 == 1.0 && d2 == 0.0;
    const bool stable = g2 != 0.0 && (!d.has_inv || (std::fabs(d.rho) <= 1.0 && std::fabs(den) > 1e-8));
    d.kind = identity ? 0 : (stable ? 1 : 2);
  }
}

const SOps* sops_for(dwf_lattice* L, double m, dwf_status* st) {
  *st = DWF_OK;
  for (auto& o : L->sops)
    if (o.m == m) return &o;
  const int n = L->Ls;
  // Q on the P+ half is the down-shift, on the P- half the up-shift.
  Mat up, dn;
  shifts(n, m, &up, &dn);
  const Mat I = eye(n);
  const double b = L->p.b, c = L->p.c, w = 4.0 - L->p.M5;
  std::vector<double> host((size_t)SOps::NKIND * 2 * n * n);
  for (int chi = 0; chi < 2; ++chi) {
    const Mat& Q = chi == 0 ? dn : up;
    Mat B = lin(b, I, c, Q);
    Mat A = lin(w, B, 1.0, lin(1.0, I, -1.0, Q));
    Mat Ai, Bi;
    if (!inverse(A, n, &Ai) || !inverse(B, n, &Bi)) {
      *st = fail(L, DWF_ERR_INVALID_ARG, "singular fifth-dimension operator for this mass");
      return nullptr;
    }
    Mat E1 = mul(B, Ai, n), E0 = mul(A, Bi, n);
    const Mat* mats[SOps::NKIND];
    Mat AT = transpose(A, n), AiT = transpose(Ai, n), BT = transpose(B, n), BiT = transpose(Bi, n);
    Mat E1T = transpose(E1, n), E0T = transpose(E0, n);
    mats[SOps::A] = &A;
    mats[SOps::AT] = &AT;
    mats[SOps::AINV] = &Ai;
    mats[SOps::AINVT] = &AiT;
    mats[SOps::B] = &B;
    mats[SOps::BT] = &BT;
    mats[SOps::BINV] = &Bi;
    mats[SOps::BINVT] = &BiT;
    mats[SOps::E1] = &E1;
    mats[SOps::E1T] = &E1T;
    mats[SOps::E0] = &E0;
    mats[SOps::E0T] = &E0T;
    for (int k = 0; k < SOps::NKIND; ++k)
      std::memcpy(host.data() + ((size_t)k * 2 + chi) * n * n, mats[k]->data(), sizeof(double) * n * n);
  }
  std::vector<float> hf(host.begin(), host.end());
  SOps o;
  o.m = m;
  fifth_descriptors(L->p, n, m, o.desc);
  if (cudaMalloc(&o.d64, host.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&o.d32, hf.size() * sizeof(float)) != cudaSuccess) {
    *st = fail(L, DWF_ERR_OOM, "s-op matrices");
    return nullptr;
  }
  if (cudaMemcpy(o.d64, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(o.d32, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    *st = fail(L, DWF_ERR_CUDA, "s-op upload");
    return nullptr;
  }
  L->sops.push_back(o);
  return &L->sops.back();
}

// ---------------------------------------------------------------- packing kernels

struct Geo {
  int X, Y, Z, T;
  long Vh;
};

__device__ __forceinline__ long full_site(const Geo& g, long h, int parity, int* xyzt) {
  const int Xh = g.X / 2;
  long rest = h / Xh;
  const int xh = (int)(h - rest * Xh);
  const int y = (int)(rest % g.Y);
  rest /= g.Y;
  const int z = (int)(rest % g.Z);
  const int t = (int)(rest / g.Z);
  const int x = 2 * xh + ((parity + y + z + t) & 1);
  if (xyzt) {
    xyzt[0] = x;
    xyzt[1] = y;
    xyzt[2] = z;
    xyzt[3] = t;
  }
  return (((long)t * g.Z + z) * g.Y + y) * g.X + x;
}

template <class S>
__global__ void pack_kernel(const double2* __restrict__ bnd, Geo g, int Ls, int Lh, int parity, FieldRef<S> out) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Vh * Ls) return;
  const long h = q / Ls;
  const int s = (int)(q - h * Ls);
  const long n = full_site(g, h, parity, nullptr);
  const long V4 = 2 * g.Vh;
  typename Store<S>::calc_t v[24];
  const double2* src = bnd + ((long)s * V4 + n) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 a = src[k];
    v[2 * k] = (typename Store<S>::calc_t)a.x;
    v[2 * k + 1] = (typename Store<S>::calc_t)a.y;
  }
  store_spinor<S>(out, h, s, Lh, v);
}

template <class S>
__global__ void unpack_kernel(CFieldRef<S> in, Geo g, int Ls, int Lh, int parity, double2* __restrict__ bnd,
                              int zero_other) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Vh * Ls) return;
  const long h = q / Ls;
  const int s = (int)(q - h * Ls);
  const long n = full_site(g, h, parity, nullptr);
  const long V4 = 2 * g.Vh;
  typename Store<S>::calc_t v[24];
  load_spinor<S>(in, h, s, Lh, v);
  double2* dst = bnd + ((long)s * V4 + n) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
  if (zero_other) {
    const long n2 = full_site(g, h, 1 - parity, nullptr);
    double2* d2 = bnd + ((long)s * V4 + n2) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) d2[k] = make_double2(0.0, 0.0);
  }
}

template <class S>
__global__ void pack_gauge_kernel(const double2* __restrict__ U, Geo g, int bc_t, S* __restrict__ out0,
                                  S* __restrict__ out1) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * g.Vh * 8) return;
  const int d = (int)(q % 8);
  const long hp = q / 8;
  const int parity = (int)(hp / g.Vh);
  const long h = hp - (long)parity * g.Vh;
  int c[4];
  full_site(g, h, parity, c);
  const int mu = d & 3;
  const long V4 = 2 * g.Vh;
  const int ext[4] = {g.X, g.Y, g.Z, g.T};
  double phase = 1.0;
  int src[4] = {c[0], c[1], c[2], c[3]};
  if (d >= 4) {
    src[mu] -= 1;
    if (src[mu] < 0) {
      src[mu] += ext[mu];
      if (mu == 3 && bc_t < 0) phase = -1.0;
    }
  } else if (mu == 3 && c[3] == g.T - 1 && bc_t < 0) {
    phase = -1.0;
  }
  const long n = (((long)src[3] * g.Z + src[2]) * g.Y + src[1]) * g.X + src[0];
  const double2* u = U + ((long)mu * V4 + n) * 9;
  S* o = (parity == 0 ? out0 : out1) + (h * 8 + d) * 18;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double2 v = d < 4 ? u[a * 3 + b] : make_double2(u[b * 3 + a].x, -u[b * 3 + a].y);
      o[2 * (a * 3 + b)] = (S)(phase * v.x);
      o[2 * (a * 3 + b) + 1] = (S)(phase * v.y);
    }
}

static Geo geo(const dwf_lattice* L) { return Geo{L->X, L->Y, L->Z, L->T, L->Vh}; }

template <class S> static FieldRef<S> fref(Field f) { return FieldRef<S>{reinterpret_cast<S*>(f.v), f.norm}; }
template <class S> static CFieldRef<S> cfref(Field f) {
  return CFieldRef<S>{reinterpret_cast<const S*>(f.v), f.norm};
}

dwf_status launch_pack(dwf_lattice* L, const void* bnd, int parity, Field out) {
  const long n = L->Vh * L->Ls;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const double2* b = reinterpret_cast<const double2*>(bnd);
  const int Ls = L->Ls, Lh = L->Lh;
  switch (out.prec) {
    case DWF_F64: pack_kernel<double><<<blocks, 256, 0, L->stream>>>(b, geo(L), Ls, Lh, parity, fref<double>(out)); break;
    case DWF_F32: pack_kernel<float><<<blocks, 256, 0, L->stream>>>(b, geo(L), Ls, Lh, parity, fref<float>(out)); break;
    case DWF_F16: pack_kernel<__half><<<blocks, 256, 0, L->stream>>>(b, geo(L), Ls, Lh, parity, fref<__half>(out)); break;
  }
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status launch_unpack(dwf_lattice* L, Field in, int parity, void* bnd, bool zero_other) {
  const long n = L->Vh * L->Ls;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  double2* b = reinterpret_cast<double2*>(bnd);
  const int Ls = L->Ls, Lh = L->Lh;
  switch (in.prec) {
    case DWF_F64: unpack_kernel<double><<<blocks, 256, 0, L->stream>>>(cfref<double>(in), geo(L), Ls, Lh, parity, b, zero_other); break;
    case DWF_F32: unpack_kernel<float><<<blocks, 256, 0, L->stream>>>(cfref<float>(in), geo(L), Ls, Lh, parity, b, zero_other); break;
    case DWF_F16: unpack_kernel<__half><<<blocks, 256, 0, L->stream>>>(cfref<__half>(in), geo(L), Ls, Lh, parity, b, zero_other); break;
  }
  DWF_LAUNCHED(L);
  return DWF_OK;
}

// [Vh][8][18] -> [8][Vh][20] (the FP32 direction-major copy)
__global__ void links_direction_major(const float* __restrict__ src, float* __restrict__ dst, long Vh) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Vh * 8) return;
  const long h = q >> 3;
  const int d = (int)(q & 7);
  const float* s = src + (h * 8 + d) * 18;
  float* o = dst + ((long)d * Vh + h) * 20;
#pragma unroll
  for (int e = 0; e < 18; ++e) o[e] = s[e];
  o[18] = 0.f;
  o[19] = 0.f;
}

dwf_status launch_pack_gauge(dwf_lattice* L, const void* U) {
  const size_t per = (size_t)L->Vh * 8 * 18;
  const size_t esz[3] = {8, 4, 2};
  for (int p = 0; p < 3; ++p)
    for (int par = 0; par < 2; ++par) {
      if (!L->links[p][par]) {
        cudaError_t e = cudaMalloc(&L->links[p][par], per * esz[p]);
        if (e != cudaSuccess) return cuda_check(L, e, "gauge copy");
      }
    }
  const long n = 2 * L->Vh * 8;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const double2* u = reinterpret_cast<const double2*>(U);
  pack_gauge_kernel<double><<<blocks, 256, 0, L->stream>>>(u, geo(L), L->p.bc_t, (double*)L->links[0][0], (double*)L->links[0][1]);
  pack_gauge_kernel<float><<<blocks, 256, 0, L->stream>>>(u, geo(L), L->p.bc_t, (float*)L->links[1][0], (float*)L->links[1][1]);
  pack_gauge_kernel<__half><<<blocks, 256, 0, L->stream>>>(u, geo(L), L->p.bc_t, (__half*)L->links[2][0], (__half*)L->links[2][1]);
  counted(L, 2);
  DWF_LAUNCHED(L);
  for (int par = 0; par < 2; ++par) {
    if (!L->links_dm[par]) {
      cudaError_t e = cudaMalloc(&L->links_dm[par], (size_t)L->Vh * 8 * 20 * sizeof(float));
      if (e != cudaSuccess) return cuda_check(L, e, "gauge copy (direction-major)");
    }
    links_direction_major<<<(unsigned)((L->Vh * 8 + 255) / 256), 256, 0, L->stream>>>(
        (const float*)L->links[1][par], L->links_dm[par], L->Vh);
    DWF_LAUNCHED(L);
  }
  return DWF_OK;
}

// ---------------------------------------------------------------- instrumentation

dwf_status timing_begin(dwf_lattice* L, cudaEvent_t* a, cudaEvent_t* b) {
  for (cudaEvent_t* e : {a, b}) {
    if (!L->ev_free.empty()) {
      *e = L->ev_free.back();
      L->ev_free.pop_back();
    } else {
      DWF_CUDA(L, cudaEventCreate(e));
    }
  }
  DWF_CUDA(L, cudaEventRecord(*a, L->stream));
  return DWF_OK;
}

void timing_end(dwf_lattice* L, int prec, double bytes, cudaEvent_t a, cudaEvent_t b) {
  cudaEventRecord(b, L->stream);
  L->pending.push_back({prec, bytes, a, b});
}

dwf_status timing_drain(dwf_lattice* L) {
  for (auto& p : L->pending) {
    float ms = 0.f;
    DWF_CUDA(L, cudaEventElapsedTime(&ms, p.a, p.b));
    L->t_ms[p.prec] += ms;
    L->t_bytes[p.prec] += p.bytes;
    L->t_n[p.prec] += 1;
    L->ev_free.push_back(p.a);
    L->ev_free.push_back(p.b);
  }
  L->pending.clear();
  return DWF_OK;
}

// ---------------------------------------------------------------- internal operators

// out_e/out_o = D(m) x or D(m)^+ x on FP64 fields (whole lattice as two parities).
dwf_status apply_D(dwf_lattice* L, const SOps* ops, bool dag, Field xe, Field xo, Field oe, Field oo) {
  const bool shamir = (L->p.b == 1.0 && L->p.c == 0.0);
  Field in[2] = {xe, xo};
  Field out[2] = {oe, oo};
  if (!dag) {
    // out_p = A x_p - 1/2 Dhop (B x_{1-p})
    Field t[2] = {xe, xo};
    if (!shamir) {
      DWF_TRY(field_alloc(L, "applyD.te", DWF_F64, &t[0]));
      DWF_TRY(field_alloc(L, "applyD.to", DWF_F64, &t[1]));
      for (int p = 0; p < 2; ++p) DWF_TRY(launch_sop(L, in[p], t[p], ops, SOps::B, 1.0, nullptr, 0.0));
    }
    for (int p = 0; p < 2; ++p) {
      HopCall c;
      c.out_parity = p;
      c.dag = 0;
      c.in = t[1 - p];
      c.out = out[p];
      c.x = in[p];
      c.has_x = true;
      c.ex = SOps::A;
      c.ops = ops;
      c.scale = -0.5;
      DWF_TRY(launch_hop(L, c));
    }
  } else {
    // out_p = A^+ x_p - 1/2 B^+ Dhop^+ x_{1-p} = B^+ (E0^+ x_p - 1/2 Dhop^+ x_{1-p})
    for (int p = 0; p < 2; ++p) {
      HopCall c;
      c.out_parity = p;
      c.dag = 1;
      c.in = in[1 - p];
      c.out = out[p];
      c.x = in[p];
      c.has_x = true;
      c.ex = shamir ? SOps::AT : SOps::E0T;
      c.eout = shamir ? SOps::NKIND : SOps::BT;
      c.ops = ops;
      c.scale = -0.5;
      DWF_TRY(launch_hop(L, c));
    }
  }
  return DWF_OK;
}

// out_e = M_pc x_e (or its adjoint), FP64.  u_o is an odd-parity temporary.
dwf_status apply_Mpc_internal(dwf_lattice* L, const SOps* ops, bool dag, Field xe, Field oe) {
  Field u, t;
  DWF_TRY(field_alloc(L, "Mpc.u", xe.prec, &u));
  HopCall c1, c2;
  c1.ops = c2.ops = ops;
  if (!dag) {
    DWF_TRY(field_alloc(L, "Mpc.t", xe.prec, &t));
    DWF_TRY(launch_sop(L, xe, t, ops, SOps::B, 1.0, nullptr, 0.0));
    c1.out_parity = 1; c1.dag = 0; c1.in = t; c1.out = u; c1.eout = SOps::E1;
    c2.out_parity = 0; c2.dag = 0; c2.in = u; c2.out = oe; c2.x = xe; c2.has_x = true;
    c2.ex = SOps::A; c2.scale = -0.25;
  } else {
    c1.out_parity = 1; c1.dag = 1; c1.in = xe; c1.out = u; c1.eout = SOps::E1T;
    c2.out_parity = 0; c2.dag = 1; c2.in = u; c2.out = oe; c2.x = xe; c2.has_x = true;
    c2.ex = SOps::E0T; c2.eout = SOps::BT; c2.scale = -0.25;  // A^+ x - 1/4 B^+ Dhop^+ u = B^+ (E0^+ x - 1/4 Dhop^+ u)
  }
  DWF_TRY(launch_hop(L, c1));
  DWF_TRY(launch_hop(L, c2));
  return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

// ---------------------------------------------------------------- C ABI

extern "C" {

const char* dwf_last_error(dwf_lattice_t h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

dwf_status dwf_create_lattice(const dwf_params* p, void* stream, dwf_lattice_t* out) {
  if (!p || !out) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: null argument");
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (p->dims[i] < 2 || (p->dims[i] & 1))
      return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: every extent must be even and >= 2");
  if (p->Ls < 1 || p->Ls > kMaxLs) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: Ls must be in [1, 64]");
  if (p->bc_t != 1 && p->bc_t != -1) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: bc_t must be +1 or -1");
  if (!std::isfinite(p->M5) || !std::isfinite(p->b) || !std::isfinite(p->c))
    return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: non-finite parameter");
  const long V4 = (long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  if (V4 / 2 * p->Ls > (1L << 31) - 1) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_create_lattice: lattice too large");
  dwf_lattice* L = new dwf_lattice();
  L->p = *p;
  L->X = p->dims[0];
  L->Y = p->dims[1];
  L->Z = p->dims[2];
  L->T = p->dims[3];
  L->V4 = V4;
  L->Vh = V4 / 2;
  L->Ls = p->Ls;
  L->Lh = (p->Ls + 1) / 2;
  L->stream = reinterpret_cast<cudaStream_t>(stream);
  // neighbour tables
  std::vector<int> nb((size_t)8 * L->Vh);
  for (int par = 0; par < 2; ++par) {
    build_neighbour_table(L->X, L->Y, L->Z, L->T, par, nb.data());
    cudaError_t e = cudaMalloc(&L->nbr[par], nb.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(L->nbr[par], nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      dwf_status st = cuda_check(nullptr, e, "neighbour table");
      dwf_destroy_lattice(L);
      return st;
    }
  }
  cudaError_t e = cudaMalloc(&L->partials, 2 * (size_t)kPartials * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->scal, kScalars * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&L->hscal, kScalars * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(L->scal, 0, kScalars * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(L->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    dwf_status st = cuda_check(nullptr, e, "lattice scratch");
    dwf_destroy_lattice(L);
    return st;
  }
  *out = L;
  return DWF_OK;
}

dwf_status dwf_destroy_lattice(dwf_lattice_t L) {
  if (!L) return DWF_OK;
  cudaStreamSynchronize(L->stream);
  for (int i = 0; i < 2; ++i) cudaFree(L->nbr[i]);
  for (int p = 0; p < 3; ++p)
    for (int i = 0; i < 2; ++i) cudaFree(L->links[p][i]);
  for (int i = 0; i < 2; ++i) cudaFree(L->links_dm[i]);
  for (auto& o : L->sops) {
    cudaFree(o.d64);
    cudaFree(o.d32);
  }
  for (auto& kv : L->ws) cudaFree(kv.second.p);
  cudaFree(L->partials);
  cudaFree(L->scal);
  cudaFree(L->dev_err);
  cudaFreeHost(L->hscal);
  for (auto& p : L->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : L->ev_free) cudaEventDestroy(e);
  delete L;
  return DWF_OK;
}

dwf_status dwf_set_kernel_timing(dwf_lattice_t L, int enable) {
  if (!L) return fail(L, DWF_ERR_INVALID_ARG, "dwf_set_kernel_timing: null handle");
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  DWF_TRY(timing_drain(L));
  L->timing = enable != 0;
  for (int p = 0; p < 3; ++p) {
    L->t_ms[p] = L->t_bytes[p] = 0.0;
    L->t_n[p] = 0;
  }
  return DWF_OK;
}

dwf_status dwf_get_kernel_time(dwf_lattice_t L, dwf_prec prec, double* ms, long long* launches, double* bytes) {
  if (!L || prec < DWF_F64 || prec > DWF_F16) return fail(L, DWF_ERR_INVALID_ARG, "dwf_get_kernel_time: bad argument");
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  DWF_TRY(timing_drain(L));
  if (ms) *ms = L->t_ms[prec];
  if (launches) *launches = L->t_n[prec];
  if (bytes) *bytes = L->t_bytes[prec];
  return DWF_OK;
}

dwf_status dwf_set_wait_limit(dwf_lattice_t L, long long polls) {
  if (!L) return fail(L, DWF_ERR_INVALID_ARG, "dwf_set_wait_limit: null handle");
  L->wait_limit = polls < 0 ? kHopWaitLimit : (long)polls;
  return DWF_OK;
}

dwf_status dwf_set_fp64_arithmetic(dwf_lattice_t L, int mode) {
  if (!L) return fail(L, DWF_ERR_INVALID_ARG, "dwf_set_fp64_arithmetic: null handle");
  if (mode != 0 && mode != 1) return fail(L, DWF_ERR_INVALID_ARG, "dwf_set_fp64_arithmetic: mode must be 0 or 1");
  L->fp64_arith = mode;
  return DWF_OK;
}

dwf_status dwf_get_launch_count(dwf_lattice_t L, long long* launches) {
  if (!L || !launches) return fail(L, DWF_ERR_INVALID_ARG, "dwf_get_launch_count: null argument");
  *launches = L->launches;
  return DWF_OK;
}

dwf_status dwf_set_gauge(dwf_lattice_t L, const void* U) {
  if (!L || !U) return fail(L, DWF_ERR_INVALID_ARG, "dwf_set_gauge: null argument");
  DWF_TRY(launch_pack_gauge(L, U));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  L->gauge_set = true;
  return DWF_OK;
}

static dwf_status apply_full(dwf_lattice_t L, double m, const void* in, void* out, int mode) {
  if (!L || !in || !out) return fail(L, DWF_ERR_INVALID_ARG, "apply: null argument");
  if (in == out) return fail(L, DWF_ERR_INVALID_ARG, "apply: in and out must not alias");
  if (!std::isfinite(m)) return fail(L, DWF_ERR_INVALID_ARG, "apply: non-finite mass");
  dwf_status st;
  const SOps* ops = sops_for(L, m, &st);
  if (!ops) return st;
  Field xe, xo, ye, yo;
  DWF_TRY(field_alloc(L, "apply.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "apply.xo", DWF_F64, &xo));
  DWF_TRY(field_alloc(L, "apply.ye", DWF_F64, &ye));
  DWF_TRY(field_alloc(L, "apply.yo", DWF_F64, &yo));
  DWF_TRY(launch_pack(L, in, 0, xe));
  DWF_TRY(launch_pack(L, in, 1, xo));
  if (mode == 0 || mode == 1) {
    DWF_TRY(apply_D(L, ops, mode == 1, xe, xo, ye, yo));
  } else {
    DWF_TRY(apply_D(L, ops, false, xe, xo, ye, yo));
    DWF_TRY(apply_D(L, ops, true, ye, yo, xe, xo));
    std::swap(xe, ye);
    std::swap(xo, yo);
  }
  DWF_TRY(launch_unpack(L, ye, 0, out, false));
  DWF_TRY(launch_unpack(L, yo, 1, out, false));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}

dwf_status dwf_apply_M(dwf_lattice_t L, double m, const void* in, void* out) { return apply_full(L, m, in, out, 0); }
dwf_status dwf_apply_Mdag(dwf_lattice_t L, double m, const void* in, void* out) { return apply_full(L, m, in, out, 1); }
dwf_status dwf_apply_MdagM(dwf_lattice_t L, double m, const void* in, void* out) { return apply_full(L, m, in, out, 2); }

dwf_status dwf_apply_Mpc(dwf_lattice_t L, double m, int dag, const void* in, void* out) {
  if (!L || !in || !out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc: null argument");
  if (in == out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc: in and out must not alias");
  dwf_status st;
  const SOps* ops = sops_for(L, m, &st);
  if (!ops) return st;
  Field xe, ye;
  DWF_TRY(field_alloc(L, "apply.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "apply.ye", DWF_F64, &ye));
  DWF_TRY(launch_pack(L, in, 0, xe));
  DWF_TRY(apply_Mpc_internal(L, ops, dag != 0, xe, ye));
  DWF_TRY(launch_unpack(L, ye, 0, out, true));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}

}  // extern "C"
