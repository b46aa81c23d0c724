// Order dispatch of the operator kernels (instantiated per order and precision
// in ax_n<N>_f32.cu / ax_n<N>_f64.cu; declared extern here so that this unit
// does not compile every kernel again).
#include "ax_impl.cuh"

namespace fnpf {

#define FNPF_EXTERN_AX(T, N)                                                                              \
  extern template cudaError_t launch_ax_n<T, N>(const Geom&, const Tables<T>&, const AxPtrs<T>&, int, int, \
                                                cudaStream_t);
#define FNPF_EXTERN_AX_ORDER(N) FNPF_EXTERN_AX(double, N) FNPF_EXTERN_AX(float, N)
FNPF_EXTERN_AX_ORDER(2)
FNPF_EXTERN_AX_ORDER(3)
FNPF_EXTERN_AX_ORDER(4)
FNPF_EXTERN_AX_ORDER(5)
FNPF_EXTERN_AX_ORDER(6)
FNPF_EXTERN_AX_ORDER(7)
FNPF_EXTERN_AX_ORDER(8)
FNPF_EXTERN_AX_ORDER(9)
#undef FNPF_EXTERN_AX_ORDER
#undef FNPF_EXTERN_AX

template <typename T>
static cudaError_t dispatch(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, int variant,
                            cudaStream_t s) {
  switch (g.n) {
    case 2: return launch_ax_n<T, 2>(g, t, a, mode, variant, s);
    case 3: return launch_ax_n<T, 3>(g, t, a, mode, variant, s);
    case 4: return launch_ax_n<T, 4>(g, t, a, mode, variant, s);
    case 5: return launch_ax_n<T, 5>(g, t, a, mode, variant, s);
    case 6: return launch_ax_n<T, 6>(g, t, a, mode, variant, s);
    case 7: return launch_ax_n<T, 7>(g, t, a, mode, variant, s);
    case 8: return launch_ax_n<T, 8>(g, t, a, mode, variant, s);
    case 9: return launch_ax_n<T, 9>(g, t, a, mode, variant, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_apply(const Geom& g, const Tables<T>& t, const T* eta, const T* xI, const T* xs, T* yI, T* ys,
                         T* ring, int variant, cudaStream_t s, const int* skip, const Epilogue<T>* ep) {
  AxPtrs<T> a{eta, xI, xs, yI, ys, ring, skip, nullptr};
  if (ep) {
    if (ys) return cudaErrorInvalidValue;
    a.ep = *ep;
  }
  return dispatch<T>(g, t, a, AX_APPLY, variant, s);
}

template <typename T>
cudaError_t launch_diag(const Geom& g, const Tables<T>& t, const T* eta, T* dI, T* ds, T* ring, cudaStream_t s) {
  AxPtrs<T> a{eta, nullptr, nullptr, dI, ds, ring, nullptr, nullptr};
  return dispatch<T>(g, t, a, AX_DIAG, 1, s);
}

int apply_variants(int n, int dim) { return dim == 2 ? 1 : kCtaVariants; }

cudaError_t ax_prepare(int n) {
  Geom g{};
  g.n = n;
  const Tables<double> t{};
  const Tables<float> t32{};
  const AxPtrs<double> a{};
  const AxPtrs<float> a32{};
  cudaError_t e = dispatch<double>(g, t, a, AX_INIT, 0, nullptr);
  return e == cudaSuccess ? dispatch<float>(g, t32, a32, AX_INIT, 0, nullptr) : e;
}

int cta_columns(int n, int dim, int variant) {
  if (dim == 2) return (128 + n - 1) / n;
  if (variant < 0 || variant >= kCtaVariants) return 0;
  switch (n) {
    case 2: return CtaChoices<2>::c[variant];
    case 3: return CtaChoices<3>::c[variant];
    case 4: return CtaChoices<4>::c[variant];
    case 5: return CtaChoices<5>::c[variant];
    case 6: return CtaChoices<6>::c[variant];
    case 7: return CtaChoices<7>::c[variant];
    case 8: return CtaChoices<8>::c[variant];
    case 9: return CtaChoices<9>::c[variant];
    default: return 0;
  }
}

int64_t geom_points(const Geom& g) { return (int64_t)g.nz * g.n_ecol * g.n * g.lines; }

template <typename T>
cudaError_t launch_geom(const Geom& g, const Tables<T>& t, const T* eta, T* G, cudaStream_t s) {
  AxPtrs<T> a{eta, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, G};
  return dispatch<T>(g, t, a, AX_GEOM, 1, s);
}

template <typename T>
cudaError_t launch_apply_g(const Geom& g, const Tables<T>& t, const T* G, const T* xI, const T* xs, T* yI, T* ys,
                           T* ring, int variant, cudaStream_t s, const int* skip, const Epilogue<T>* ep) {
  AxPtrs<T> a{nullptr, xI, xs, yI, ys, ring, skip, const_cast<T*>(G)};
  if (ep) {
    if (ys) return cudaErrorInvalidValue;
    a.ep = *ep;
  }
  return dispatch<T>(g, t, a, AX_APPLY_G, variant, s);
}

template cudaError_t launch_geom<double>(const Geom&, const Tables<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_geom<float>(const Geom&, const Tables<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_apply_g<double>(const Geom&, const Tables<double>&, const double*, const double*,
                                            const double*, double*, double*, double*, int, cudaStream_t, const int*,
                                            const Epilogue<double>*);
template cudaError_t launch_apply_g<float>(const Geom&, const Tables<float>&, const float*, const float*,
                                           const float*, float*, float*, float*, int, cudaStream_t, const int*,
                                           const Epilogue<float>*);

template cudaError_t launch_apply<double>(const Geom&, const Tables<double>&, const double*, const double*,
                                          const double*, double*, double*, double*, int, cudaStream_t,
                                          const int*, const Epilogue<double>*);
template cudaError_t launch_apply<float>(const Geom&, const Tables<float>&, const float*, const float*, const float*,
                                         float*, float*, float*, int, cudaStream_t, const int*,
                                         const Epilogue<float>*);
template cudaError_t launch_diag<double>(const Geom&, const Tables<double>&, const double*, double*, double*,
                                         double*, cudaStream_t);
template cudaError_t launch_diag<float>(const Geom&, const Tables<float>&, const float*, float*, float*, float*,
                                        cudaStream_t);

}  // namespace fnpf
