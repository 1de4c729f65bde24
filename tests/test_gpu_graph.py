"""fv_decode is capturable: no host synchronisation and no allocation
inside, so a whole decode (prep, order, forward, backtrack -- or every
FLASH level) can be recorded once into a CUDA graph and replayed.  Replays
on new emission scores written into the same input buffer must give the
oracle's paths and scores."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    import paper_2510_19301_gb300 as fv
    fv._lib.load(build_if_missing=True)
    return fv


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


@pytest.mark.parametrize("mode,kw,K", [("vanilla", {}, 256), ("flash", {"P": 4}, 256),
                                       ("flash", {"P": 4, "mem_budget": 64 * 256 * 2}, 256),
                                       ("vanilla", {}, 2048), ("beam", {"B": 16, "P": 0}, 64),
                                       ("beam", {"B": 16, "P": 2}, 64)])
def test_decode_graph_replay(fv, mode, kw, K):
    rng = np.random.default_rng(K + len(kw))
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 5] + list(rng.integers(2, 60 if K > 1024 else 200, 6))
    total = int(np.sum(lengths))
    m = fv.Model(log_pi, logA)
    E_dev = torch.zeros(total * K, dtype=torch.float32, device="cuda")
    b = fv.Batch(lengths, E=E_dev, models=[m])
    dec = fv.Decoder([m], b, mode=mode, **kw)
    stream = torch.cuda.Stream()
    # warm-up outside capture (first calls set kernel attributes)
    with torch.cuda.stream(stream):
        dec.launch(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        dec.launch(stream)
    hmm = oracle.HMM(log_pi, logA)
    for rep in range(2):
        E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
        E_dev.copy_(torch.from_numpy(np.concatenate(E_list)).view(-1))
        graph.replay()
        torch.cuda.synchronize()
        assert dec.device_status() == 0
        paths, scores = dec.paths.cpu().numpy(), dec.scores.cpu().numpy()
        if mode == "beam" and kw["P"] == 0:
            ref = [oracle.beam(hmm, e, kw["B"])[:2] for e in E_list]
        elif mode == "beam":
            ref = [oracle.flash_bs(hmm, e, kw["P"], kw["B"])[:2] for e in E_list]
        else:
            ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
        off = 0
        for i, (p, s) in enumerate(ref):
            T = lengths[i]
            assert np.array_equal(paths[off:off + T], p), f"{mode} rep {rep} seq {i}"
            assert bits(scores[i]) == bits(s), f"{mode} rep {rep} seq {i}"
            off += T
