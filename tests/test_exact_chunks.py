"""The arithmetic the INT8 layers' tensor-core kernels rely on, checked on the
CPU: the INT8 network's dot products (Sec. II-B's dense layers in the INT8
reading: u8 activations or s8 priors times s8 weights, exact integer sums)
run as bf16 MMAs with FP32 accumulation, so

  - every operand must be exact in bf16: the integers -128..255 have at most
    8 significant bits, and bf16 keeps 8;
  - every FP32 partial sum must be exact whatever order the tensor core adds
    in: with K cut into chunks of 256 each partial sum is an integer of
    magnitude at most 256 * 255 * 127 < 2^23;
  - without the chunks (K = 4096 in one accumulator) the sums reach 2^27 and
    FP32 loses their low bits, which is why the kernels convert each chunk's
    accumulator to int32 and add the chunks as integers."""
import numpy as np

CHUNK = 256


def _bf16(x):
    """Round-to-nearest-even float32 -> bf16 -> float32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _fp32_sum(terms, order):
    acc = np.float32(0.0)
    for i in order:
        acc = np.float32(acc + np.float32(terms[i]))
    return acc


def test_int8_operands_are_exact_in_bf16():
    v = np.arange(-128, 256, dtype=np.float32)
    assert np.array_equal(_bf16(v), v)
    # the first integer that bf16 cannot hold
    assert _bf16(np.float32(257.0)) != 257.0


def test_chunk_sums_are_exact_in_any_order():
    rng = np.random.default_rng(5)
    # the worst case (every product 255 * 127 or 255 * -127), then random ones
    cases = [np.full(CHUNK, 255 * 127), np.full(CHUNK, -255 * 127)]
    cases += [rng.integers(0, 256, CHUNK) * rng.integers(-127, 128, CHUNK) for _ in range(20)]
    assert CHUNK * 255 * 127 < 2 ** 23
    for terms in cases:
        exact = int(np.sum(terms.astype(np.int64)))
        for _ in range(5):
            assert int(_fp32_sum(terms, rng.permutation(CHUNK))) == exact
        # partial sums of any prefix stay integers below 2^23
        assert np.max(np.abs(np.cumsum(terms.astype(np.int64)))) < 2 ** 23


def test_chunks_added_as_integers_give_the_dot_product():
    rng = np.random.default_rng(7)
    K = 4096
    x = rng.integers(0, 256, K)
    w = rng.integers(-127, 128, K)
    terms = x * w
    chunks = [int(_fp32_sum(terms[c:c + CHUNK], range(CHUNK))) for c in range(0, K, CHUNK)]
    assert sum(chunks) == int(np.dot(x.astype(np.int64), w.astype(np.int64)))


def test_one_accumulator_over_4096_products_is_not_exact():
    # 4096 products of 255 * 127 (odd) plus one of 1: past 2^24 an FP32 sum
    # rounds to even, so a single accumulator drops units that int32 keeps
    terms = np.concatenate([np.full(4096, 255 * 127), [1]])
    exact = int(np.sum(terms))
    assert exact > 2 ** 24
    assert int(_fp32_sum(terms, range(terms.size))) != exact
