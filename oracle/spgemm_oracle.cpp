// CPU oracle for C = A * B (test infrastructure, not part of the library).
//
// Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg load
// this file's shared object.  It shares no code, header or helper with the
// CUDA library; both sides are fed the same arrays by the seeded generators.
//
// What it computes: the plain definition of the sparse product (Sec. 2.2,
// Gustavson's row-by-row formulation, Fig. 1): for every selected row i of A,
// for every a_ik in ascending k, for every b_kj in row k of B,
// acc[j] += a_ik * b_kj, with an ordered std::map as the sparse accumulator;
// the row of C is the map in key order.  The structure is symbolic (Sec. 2.2,
// symbolic phase): an entry whose value cancels to zero is kept.
//
// Precision: FP64 accumulation for FP32 and FP64 inputs (each product of two
// converted FP32 values is exact in FP64), wrapping 64-bit integer arithmetic
// for int64 inputs.  Compiled with -ffp-contract=off so a*b+c is two
// roundings.  Optionally also returns (|A||B|)_ij = sum_k |a_ik||b_kj|, the
// scale of the element-wise error bound the tests use.
//
// Rows are independent; with nthreads > 1 they are shared out over OpenMP
// threads, and the per-row code is unchanged.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { DT_F32 = 0, DT_F64 = 1, DT_I64 = 2 };

struct Row {
  std::vector<int32_t> col;
  std::vector<double> vf;
  std::vector<int64_t> vi;
  std::vector<double> mag;
};

struct Result {
  int dtype = 0;
  std::vector<Row> rows;
  int64_t nnz = 0;
};

inline double load_fp(const void* v, int dtype, int64_t p) {
  if (dtype == DT_F32) return (double)((const float*)v)[p];
  return ((const double*)v)[p];
}

void row_fp(int64_t i, const int64_t* arp, const int32_t* acol, const void* aval,
            const int64_t* brp, const int32_t* bcol, const void* bval, int dtype,
            bool want_mag, Row& out) {
  std::map<int32_t, double> acc;
  std::map<int32_t, double> mag;
  for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
    const int32_t k = acol[p];
    const double a = load_fp(aval, dtype, p);
    for (int64_t q = brp[k]; q < brp[k + 1]; ++q) {
      const int32_t j = bcol[q];
      const double b = load_fp(bval, dtype, q);
      acc[j] += a * b;
      if (want_mag) mag[j] += std::fabs(a) * std::fabs(b);
    }
  }
  out.col.reserve(acc.size());
  out.vf.reserve(acc.size());
  for (const auto& kv : acc) {
    out.col.push_back(kv.first);
    out.vf.push_back(kv.second);
  }
  if (want_mag)
    for (const auto& kv : mag) out.mag.push_back(kv.second);
}

void row_int(int64_t i, const int64_t* arp, const int32_t* acol, const int64_t* aval,
             const int64_t* brp, const int32_t* bcol, const int64_t* bval, bool want_mag,
             Row& out) {
  std::map<int32_t, uint64_t> acc;
  std::map<int32_t, double> mag;
  for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
    const int32_t k = acol[p];
    const uint64_t a = (uint64_t)aval[p];
    for (int64_t q = brp[k]; q < brp[k + 1]; ++q) {
      const int32_t j = bcol[q];
      acc[j] += a * (uint64_t)bval[q];
      if (want_mag) mag[j] += std::fabs((double)aval[p]) * std::fabs((double)bval[q]);
    }
  }
  for (const auto& kv : acc) {
    out.col.push_back(kv.first);
    out.vi.push_back((int64_t)kv.second);
  }
  if (want_mag)
    for (const auto& kv : mag) out.mag.push_back(kv.second);
}

}  // namespace

extern "C" {

// Computes rows `rows[0..nsel)` of A*B (all rows 0..nsel-1 when rows is NULL).
// Returns an opaque handle; free it with oracle_result_free.
void* oracle_spgemm(int64_t nsel, const int64_t* rows, const int64_t* arp, const int32_t* acol,
                    const void* aval, const int64_t* brp, const int32_t* bcol, const void* bval,
                    int dtype, int want_mag, int nthreads) {
  Result* r = new Result();
  r->dtype = dtype;
  r->rows.resize((size_t)nsel);
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
  for (int64_t s = 0; s < nsel; ++s) {
    const int64_t i = rows ? rows[s] : s;
    if (dtype == DT_I64)
      row_int(i, arp, acol, (const int64_t*)aval, brp, bcol, (const int64_t*)bval, want_mag != 0,
              r->rows[(size_t)s]);
    else
      row_fp(i, arp, acol, aval, brp, bcol, bval, dtype, want_mag != 0, r->rows[(size_t)s]);
  }
  int64_t nnz = 0;
  for (const Row& row : r->rows) nnz += (int64_t)row.col.size();
  r->nnz = nnz;
  return r;
}

int64_t oracle_result_nnz(void* h) { return ((Result*)h)->nnz; }

// row_ptr: nsel+1; col: nnz; val: nnz doubles (f32/f64) or int64 (i64); mag: nnz or NULL.
void oracle_result_copy(void* h, int64_t* row_ptr, int32_t* col, void* val, double* mag) {
  Result* r = (Result*)h;
  int64_t off = 0;
  row_ptr[0] = 0;
  for (size_t s = 0; s < r->rows.size(); ++s) {
    const Row& row = r->rows[s];
    const size_t m = row.col.size();
    if (m) {
      std::memcpy(col + off, row.col.data(), m * sizeof(int32_t));
      if (r->dtype == DT_I64)
        std::memcpy((int64_t*)val + off, row.vi.data(), m * sizeof(int64_t));
      else
        std::memcpy((double*)val + off, row.vf.data(), m * sizeof(double));
      if (mag && !row.mag.empty()) std::memcpy(mag + off, row.mag.data(), m * sizeof(double));
    }
    off += (int64_t)m;
    row_ptr[s + 1] = off;
  }
}

void oracle_result_free(void* h) { delete (Result*)h; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
