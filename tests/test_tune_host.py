"""Host side of the chunk-length tuner: candidate sets and the tuning table.

CPU-only: these entry points do no device work, so they run without a GPU
(the library only has to load). The measuring part, hmm_autotune_batched,
is covered by tests/test_gpu_tune.py.
"""
import numpy as np
import pytest

api = pytest.importorskip("paper_2003_03508_gb300.api")

SMS = 152


@pytest.fixture(autouse=True)
def _empty_table():
    try:
        api.load_library()
    except OSError as e:  # no CUDA runtime to dlopen on this host
        pytest.skip(f"cannot load the library here: {e}")
    api.tune_clear()
    yield
    api.tune_clear()


SHAPES = [
    ("tf32", 256, 32, (1 << 20) - 1),        # the batched workload
    ("fp32", 32, 32, (1 << 20) - 1),
    ("tf32", 128, 64, (1 << 22) - 1),
    ("bf16", 128, 80, (1 << 22) - 1),
    ("tf32_split", 1, 25, (1 << 20) - 1),
    ("fp32", 1, 4, 9_999),
    ("tf32", 256, 32, (1 << 24) - 64),       # 64 uneven segments
]


@pytest.mark.parametrize("prec,n_prop,K,steps", SHAPES)
def test_candidates_are_valid_and_contain_the_model_choice(prec, n_prop, K, steps):
    L0 = api.default_chunk_len(prec, n_prop, K, steps, SMS)
    assert L0 >= 64 and L0 % 64 == 0 and L0 <= 16384
    cand = api.tune_candidates(prec, n_prop, K, steps, SMS)
    cap = min(16384, -(-steps // 64) * 64)
    assert L0 in cand
    assert cand == sorted(set(cand)), cand
    assert 1 <= len(cand) <= 16
    assert all(64 <= L <= cap and L % 64 == 0 for L in cand), cand
    # the geometric neighbours of the model's choice (clamped to the range) are measured
    for j in (-2, 2):
        L = min(cap, max(64, int(L0 * 2.0 ** (0.5 * j) / 64 + 0.5) * 64))
        assert L in cand, (L, cand)


def test_candidates_short_sequences():
    # no chain steps, or fewer than one window: one candidate, the smallest chunk
    assert api.tune_candidates("tf32", 8, 32, 0, SMS) == [64]
    assert api.tune_candidates("fp32", 8, 32, 10, SMS) == [64]
    # never longer than the sequence rounded up to the 64-step window
    assert max(api.tune_candidates("fp32", 1, 4, 1000, SMS)) <= 1024


def test_candidates_reject_bad_arguments():
    for args in (("fp32", 0, 4, 100, SMS), ("fp32", 1, 0, 100, SMS), ("fp32", 1, 81, 100, SMS),
                 ("fp32", 1, 4, -1, SMS), ("fp32", 1, 4, 100, 0), (9, 1, 4, 100, SMS)):
        with pytest.raises(api.HMMError):
            api.tune_candidates(*args)
        assert api.default_chunk_len(*args) == 0


def _write(path, lines):
    path.write_text("".join(l + "\n" for l in lines))
    return path


def test_table_load_lookup_save_roundtrip(tmp_path):
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, (1 << 20) - 1) == 0
    f = _write(tmp_path / "t.txt", [
        "# comment",
        "",
        f"{SMS} 32 1 256 1 1048575 0 4096 61.25",
        f"{SMS} 32 0 32 1 1048575 4 1024 40.5",
    ])
    api.tune_load(f)
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, (1 << 20) - 1) == 4096
    assert api.tune_lookup(SMS, 32, "fp32", 32, 1, (1 << 20) - 1, runlen_min=4) == 1024
    # every field of the key matters
    assert api.tune_lookup(SMS, 32, "fp32", 32, 1, (1 << 20) - 1, runlen_min=0) == 0
    assert api.tune_lookup(148, 32, "tf32", 256, 1, (1 << 20) - 1) == 0
    assert api.tune_lookup(SMS, 32, "tf32", 256, 2, (1 << 20) - 1) == 0
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, 1 << 20) == 0
    # an entry with the same key replaces the stored one
    api.tune_load(_write(tmp_path / "u.txt", [f"{SMS} 32 1 256 1 1048575 0 8192 60.0"]))
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, (1 << 20) - 1) == 8192
    # save, clear, load: the same table
    out = tmp_path / "saved.txt"
    api.tune_save(out)
    api.tune_clear()
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, (1 << 20) - 1) == 0
    api.tune_load(out)
    assert api.tune_lookup(SMS, 32, "tf32", 256, 1, (1 << 20) - 1) == 8192
    assert api.tune_lookup(SMS, 32, "fp32", 32, 1, (1 << 20) - 1, runlen_min=4) == 1024
    rows = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert len(rows) == 2


@pytest.mark.parametrize("bad", [
    f"{SMS} 32 1 256 1 1048575 0 4000 1.0",      # not a multiple of 64
    f"{SMS} 32 1 256 1 1048575 0 32768 1.0",     # beyond 16384
    f"{SMS} 81 1 256 1 1048575 0 4096 1.0",      # K out of range
    f"{SMS} 32 7 256 1 1048575 0 4096 1.0",      # unknown precision
    f"{SMS} 32 1 0 1 1048575 0 4096 1.0",        # no proposals
    f"{SMS} 32 1 256 1 1048575 0 4096",          # a field missing
    f"{SMS} 32 1 256 1 1048575 0 4096 1.0 junk", # trailing text
    f"{SMS} 32 1 256 1 -5 0 4096 1.0",           # negative steps
    "x 32 1 256 1 1048575 0 4096 1.0",           # not a number
])
def test_table_rejects_a_malformed_file_whole(tmp_path, bad):
    f = _write(tmp_path / "bad.txt", [f"{SMS} 16 0 8 1 9999 0 512 2.0", bad])
    with pytest.raises(api.HMMError):
        api.tune_load(f)
    # the valid first line was not loaded either
    assert api.tune_lookup(SMS, 16, "fp32", 8, 1, 9999) == 0


def test_table_unreadable_and_unwritable_paths(tmp_path):
    with pytest.raises(api.HMMError):
        api.tune_load(tmp_path / "missing.txt")
    with pytest.raises(api.HMMError):
        api.tune_save(tmp_path / "no_such_dir" / "t.txt")


def test_chain_steps():
    assert api.chain_steps([0, 10]) == 9
    assert api.chain_steps([0, 0, 1, 5]) == 3


def test_table_load_survives_random_text(tmp_path):
    # arbitrary bytes never crash the loader: the file is either rejected
    # whole or (blank/comment-only) adds nothing
    rng = np.random.default_rng(0)
    alphabet = np.array(list(b"0123456789 -+.eE#x\t\n\r") + [0, 255, 10], dtype=np.uint8)
    for i in range(200):
        n = int(rng.integers(0, 300))
        data = bytes(rng.choice(alphabet, size=n)) if i % 2 else bytes(rng.integers(0, 256, size=n, dtype=np.uint8))
        f = tmp_path / f"r{i}.txt"
        f.write_bytes(data)
        try:
            api.tune_load(f)
        except api.HMMError:
            pass
    # a very long line is rejected, not truncated into a valid entry
    long_line = f"{SMS} 32 1 256 1 1048575 0 4096 " + "1" * 600 + "\n"
    f = tmp_path / "long.txt"
    f.write_text(long_line)
    with pytest.raises(api.HMMError):
        api.tune_load(f)
    api.tune_clear()
