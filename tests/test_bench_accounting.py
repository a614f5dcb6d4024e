"""The bench's algorithmic-work accounting (CPU): the roofline's numerators
count what the method must do per launch, independent of how the kernels do
it, so they are checked here against hand counts."""
import bench


W = {"dims": [1000, 800, 600], "R": 100, "J": 4096}
STATS = {"nnz_sel": 50_000, "J_u": 3000, "rows": 700, "I_mean": 800.0}


def test_df64_terms_of_gram_and_leverage_scores():
    # R(R+1)/2 pairs a row, each a double-float term of 10 float32 operations
    for phase in ("gram", "sampler"):
        bound, ops = bench.algorithmic(phase, W, STATS)
        assert bound == "alu"
        assert ops == 800.0 * 5050 * bench.DF64_TERM_OPS


def test_fast_option_counts_float32_terms():
    # one FMA a Gram term; a multiply and an FMA a leverage term
    assert bench.algorithmic("gram", W, STATS, fast=True) == ("alu", 800.0 * 5050 * 1)
    assert bench.algorithmic("sampler", W, STATS, fast=True) == ("alu", 800.0 * 5050 * 2)


def test_solve_is_one_fma_per_term():
    assert bench.algorithmic("solve", W, STATS) == ("alu", 800.0 * 100 * 100)


def test_spmm_bytes():
    # (row, value) per selected nonzero, a KRP row and offsets per distinct
    # column, one output row per touched row
    bound, b = bench.algorithmic("spmm", W, STATS)
    assert bound == "hbm"
    assert b == 50_000 * 8 + 3000 * (100 * 4 + 16) + 700 * 100 * 4


def test_replica_throughput_is_total_over_slowest():
    # one process: value = steps / seconds of its timed region
    value, total_ms = bench.replica_throughput(1, 20, 2000.0)
    assert abs(value - 10.0) < 1e-12 and total_ms == 2000.0
