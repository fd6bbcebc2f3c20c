/* Group-by of host arrays through the C ABI of libagg.so alone (no Python, no
 * PyTorch): plan the run, create a handle, aggregate host buffers, check the
 * result against invariants that hold for any correct group-by, read the run's
 * counters and release the handle.
 *
 *   cc -std=c11 -I include paper_1311_0059_gb300/examples/groupby_host.c \
 *      -L paper_1311_0059_gb300 -lagg -Wl,-rpath,paper_1311_0059_gb300 -o groupby_host
 *   ./groupby_host [rows [distinct_keys [budget_bytes]]]
 *
 * Rows draw their key uniformly from `distinct_keys` random-looking int64 keys
 * and an int64 value uniform in [0, 2^20).  Exit status: 0 when every invariant
 * holds, 1 when one fails, 2 when no GPU is usable (the plan, which needs none,
 * is printed first), 3 on any other library error.
 */
#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>

#include "agg.h"

/* SplitMix64 (Steele, Lea and Flood, 2014): the state step and its output
 * function.  The output function is a bijection of 64-bit words, so distinct
 * ranks give distinct keys. */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t next64(uint64_t* state) { return mix64(*state += 0x9E3779B97F4A7C15ull); }

static int cmp_i64(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

static uint64_t distinct_count(const int64_t* v, uint64_t n) {
  int64_t* s = malloc((n ? n : 1) * sizeof(int64_t));
  if (!s) return UINT64_MAX;
  for (uint64_t i = 0; i < n; ++i) s[i] = v[i];
  qsort(s, n, sizeof(int64_t), cmp_i64);
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i) d += (i == 0 || s[i] != s[i - 1]);
  free(s);
  return d;
}

#define CHECK(cond, what)                             \
  do {                                                \
    if (!(cond)) {                                    \
      fprintf(stderr, "invariant failed: %s\n", what); \
      failed = 1;                                     \
    }                                                 \
  } while (0)

int main(int argc, char** argv) {
  const uint64_t n = argc > 1 ? strtoull(argv[1], NULL, 10) : 1000000;
  const uint64_t domain = argc > 2 ? strtoull(argv[2], NULL, 10) : 10000;
  const size_t budget = argc > 3 ? (size_t)strtoull(argv[3], NULL, 10) : (size_t)64 << 20;
  if (domain == 0) return 3;

  agg_spec spec = {0};
  spec.ops = AGG_COUNT | AGG_SUM | AGG_MIN | AGG_MAX;
  spec.value_type = AGG_I64;
  spec.path = AGG_PATH_HASH;

  agg_plan_info plan;
  agg_status st = agg_plan(budget, &spec, NULL, n, &plan);
  if (st != AGG_OK) {
    fprintf(stderr, "agg_plan: %s\n", agg_strerror(st));
    return 3;
  }
  printf("plan: entry_bytes %" PRIu64 " table_slots %" PRIu64 " fan_out %" PRIu64 " working_bytes %" PRIu64
         " staging_bytes %" PRIu64 "\n",
         plan.entry_bytes, plan.table_slots, plan.fan_out, plan.working_bytes, plan.staging_bytes);
  fflush(stdout);

  agg_handle* h = NULL;
  st = agg_create(budget, &spec, &h);
  if (st == AGG_ERR_CUDA) {
    fprintf(stderr, "agg_create: %s (no usable GPU)\n", agg_strerror(st));
    return 2;
  }
  if (st != AGG_OK) {
    fprintf(stderr, "agg_create: %s\n", agg_strerror(st));
    return 3;
  }

  const uint64_t cap = n ? n : 1;
  int64_t* keys = malloc(cap * sizeof(int64_t));
  int64_t* vals = malloc(cap * sizeof(int64_t));
  int64_t* o_keys = malloc(cap * sizeof(int64_t));
  uint64_t* o_count = malloc(cap * sizeof(uint64_t));
  int64_t* o_sum = malloc(cap * sizeof(int64_t));
  int64_t* o_min = malloc(cap * sizeof(int64_t));
  int64_t* o_max = malloc(cap * sizeof(int64_t));
  if (!keys || !vals || !o_keys || !o_count || !o_sum || !o_min || !o_max) {
    fprintf(stderr, "out of host memory\n");
    agg_destroy(h);
    return 3;
  }
  uint64_t rng = 12345, total = 0;
  for (uint64_t i = 0; i < n; ++i) {
    keys[i] = (int64_t)mix64(next64(&rng) % domain);
    vals[i] = (int64_t)(next64(&rng) >> 44);  /* [0, 2^20) */
    total += (uint64_t)vals[i];
  }

  agg_output out = {o_keys, o_count, o_sum, o_min, o_max, cap, NULL};
  uint64_t groups = 0;
  st = agg_run_host(h, keys, vals, n, &out, &groups, NULL);
  if (st != AGG_OK) {
    fprintf(stderr, "agg_run_host: %s\n", agg_strerror(st));
    agg_destroy(h);
    return 3;
  }

  int failed = 0;
  uint64_t count_sum = 0, sum_sum = 0;
  for (uint64_t g = 0; g < groups; ++g) {
    count_sum += o_count[g];
    sum_sum += (uint64_t)o_sum[g];
    CHECK(o_count[g] >= 1, "every group has a row");
    CHECK(o_min[g] <= o_max[g] && o_min[g] >= 0 && o_max[g] < ((int64_t)1 << 20), "MIN <= MAX within the value range");
    CHECK((uint64_t)o_sum[g] >= (uint64_t)o_max[g] && (uint64_t)o_sum[g] <= o_count[g] * (uint64_t)o_max[g],
          "MAX <= SUM <= COUNT * MAX");
  }
  CHECK(count_sum == n, "sum of COUNT = rows");
  CHECK(sum_sum == total, "sum of SUM = sum of values");
  CHECK(groups == distinct_count(keys, n), "groups = distinct input keys");
  CHECK(distinct_count(o_keys, groups) == groups, "result keys are distinct");

  agg_stats s;
  if (agg_get_stats(h, &s) == AGG_OK)
    printf("run: rows %" PRIu64 " groups %" PRIu64 " levels %" PRIu64 " spilled_bytes %" PRIu64 "\n", s.n_rows,
           s.n_groups, s.levels, s.spill_bytes_written);
  agg_destroy(h);
  free(keys), free(vals), free(o_keys), free(o_count), free(o_sum), free(o_min), free(o_max);
  printf(failed ? "invariants FAILED\n" : "invariants hold\n");
  return failed;
}
