"""The Python binding's argument checks on Sorter.sort_: the C entry points
take bare pointers, so a tensor too short, of the wrong item size, strided or
on another device must be refused before any call.  Runs on CPU (a sorter
whose buffers live in host memory; every case raises before the library's
sort entry point is reached)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2207_14334_gb300 as dfr  # noqa: E402
from paper_2207_14334_gb300 import build as dfr_build  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    dfr_build.build()
    return dfr.load()


def refused(s, *args, **kw):
    with pytest.raises(ValueError):
        s.sort_(*args, **kw)


def test_key_only_arguments(lib):
    s = dfr.Sorter(dfr.DFR_U32, 64, device="cpu")
    k = torch.zeros(64, dtype=torch.int32)
    refused(s, k, n=65)                                  # beyond the capacity
    refused(s, k[:10], n=11)                             # beyond the tensor
    refused(s, k, n=-1)
    refused(s, torch.zeros(64, dtype=torch.int64))       # 8-byte items for u32 keys
    refused(s, torch.zeros(64, dtype=torch.int16))
    refused(s, k[::2])                                   # strided view
    refused(s, k, torch.zeros(64, dtype=torch.int32))    # payloads for a key-only type
    refused(s, None, n=5)
    s64 = dfr.Sorter(dfr.DFR_U64, 64, device="cpu")
    refused(s64, k)                                      # 4-byte items for u64 keys
    refused(s64, torch.zeros((8, 8), dtype=torch.int64).t())  # transposed: not contiguous


def test_kv_arguments(lib):
    s = dfr.Sorter(dfr.DFR_U64_KV, 64, device="cpu")
    k = torch.zeros(64, dtype=torch.int64)
    v = torch.zeros(64, dtype=torch.int32)
    refused(s, k)                                        # payloads missing
    refused(s, k, v[:63])                                # payloads shorter than the keys
    refused(s, k, torch.zeros(64, dtype=torch.int64))    # 8-byte payloads
    refused(s, k, v[::1].view(8, 8).t())                 # payloads not contiguous
    s32 = dfr.Sorter(dfr.DFR_U32_KV, 64, device="cpu")
    refused(s32, torch.zeros(64, dtype=torch.int32), None)


def test_other_device(lib):
    # a tensor on another device than the sorter's buffers
    s = dfr.Sorter(dfr.DFR_U32, 64, device="cpu")
    refused(s, torch.empty(64, dtype=torch.int32, device="meta"))


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # with the CUDA library absent every call raises; nothing falls back to a
    # CPU path
    monkeypatch.setattr(dfr, "LIB_PATH", str(tmp_path / "libdfr.so"))
    monkeypatch.setattr(dfr, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dfr.load()
    with pytest.raises(RuntimeError):
        dfr.dfr_workspace_bytes(dfr.DFR_U32, 1000)
    with pytest.raises(RuntimeError):
        dfr.dfr_sort_u32(0, 0, 10, 0, 0, stream=0)
