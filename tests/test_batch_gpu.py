"""Many snapshots through one call (pc_compress_batch / pc_decompress_batch)
and through the serving loop (pc_server_*): every result must be identical to
the same snapshot compressed or decompressed alone with the plain calls, and
the small ones identical to the oracle."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as b

    b.build()
    pc.load()
    return pc


def _mix(pc, seed=0, count=14):
    """Snapshots of uneven size, both generators, both dtypes, three bounds."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        n = int(round(10 ** rng.uniform(0, 5.6))) if i else 0
        dt = np.float32 if rng.random() < 0.5 else np.float64
        gen = "cosmology" if rng.random() < 0.5 else "fluid"
        pos = synth.by_name(gen, n, seed=i, dtype=dt) if n else np.zeros((0, 3), dt)
        mode = pc.PC_EB_REL if rng.random() < 0.7 else pc.PC_EB_ABS
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))
        leaf = int(rng.choice([0, 256, 4096]))
        jobs.append((pos, mode, eb, leaf))
    return jobs


def _alone(pc, pos_d, mode, eb, leaf):
    n = pos_d.shape[0]
    dt = pc.PC_F32 if pos_d.dtype == torch.float32 else pc.PC_F64
    c = pc.Compressor(n, dt, leaf_size=leaf, device=pos_d.device)
    size = c.compress(pos_d, mode, eb)
    return c.out[:size].clone()


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_batch_compress_equals_alone(pc, oracle_mod, lanes):
    dev = torch.device("cuda:0")
    jobs = _mix(pc)
    dpos = [torch.from_numpy(p).to(dev) for p, _, _, _ in jobs]
    outs = [torch.empty(pc.pc_compress_bound(p.shape[0], pc.PC_F32 if p.dtype == torch.float32 else pc.PC_F64,
                                             leaf), dtype=torch.uint8, device=dev)
            for p, (_, _, _, leaf) in zip(dpos, jobs)]
    sizes, statuses = pc.pc_compress_batch([(p, m, eb, leaf) for p, (_, m, eb, leaf) in zip(dpos, jobs)], outs,
                                           lanes=lanes)
    assert statuses == [pc.PC_OK] * len(jobs)
    for (pos, m, eb, leaf), p, o, sz in zip(jobs, dpos, outs, sizes):
        alone = _alone(pc, p, m, eb, leaf)
        assert torch.equal(o[:sz], alone)
        if pos.shape[0] <= 20_000:
            ref, _ = oracle_mod.compress(pos, oracle_mod.REL if m == pc.PC_EB_REL else oracle_mod.ABS, eb,
                                         leaf_size=leaf or 4096)
            assert o[:sz].cpu().numpy().tobytes() == ref
    # and back, in one batch
    decs = [torch.empty_like(p) for p in dpos]
    st = pc.pc_decompress_batch(outs, sizes, decs, lanes=lanes)
    assert st == [pc.PC_OK] * len(jobs)
    for p, o, sz, d in zip(dpos, outs, sizes, decs):
        if p.shape[0]:
            alone = torch.empty_like(p)
            c = pc.Compressor(p.shape[0], pc.PC_F32 if p.dtype == torch.float32 else pc.PC_F64, device=p.device)
            c.decompress(o, alone, sz)
            assert torch.equal(d, alone)


def test_batch_with_reduction_and_reordering(pc, oracle_mod):
    """Items with the reduction, the reordering, both, and autotuned leaves: each
    stream equals the same call alone, and the small ones the oracle's."""
    dev = torch.device("cuda:0")
    cfgs = [pc.config(256, reduce=True), pc.config(512, reorder=True), pc.config(300, reduce=True, reorder=True),
            pc.config(0, autotune=True, reduce=True), pc.config(4096)]
    jobs = []
    for i, cfg in enumerate(cfgs * 2):
        n = [3_000, 40_000, 250_000][i % 3]
        pos = synth.by_name("cosmology" if i % 2 else "fluid", n, seed=40 + i,
                            dtype=np.float32 if i % 4 < 2 else np.float64)
        jobs.append((pos, pc.PC_EB_REL, 1e-3, cfg))
    dpos = [torch.from_numpy(p).to(dev) for p, _, _, _ in jobs]
    outs = [torch.empty(pc.pc_compress_bound(p.shape[0], pc.PC_F32 if p.dtype == torch.float32 else pc.PC_F64, cfg),
                        dtype=torch.uint8, device=dev) for p, (_, _, _, cfg) in zip(dpos, jobs)]
    sizes, statuses = pc.pc_compress_batch([(p, m, eb, cfg) for p, (_, m, eb, cfg) in zip(dpos, jobs)], outs,
                                           lanes=4)
    assert statuses == [pc.PC_OK] * len(jobs)
    for (pos, m, eb, cfg), p, o, sz in zip(jobs, dpos, outs, sizes):
        assert torch.equal(o[:sz], _alone(pc, p, m, eb, cfg))
        if pos.shape[0] <= 3_000 and not (cfg.flags & pc.PC_FLAG_AUTOTUNE_LEAF):
            if cfg.flags & pc.PC_FLAG_BOX_REDUCTION:
                ref, _, _ = oracle_mod.compress_reduced(pos, oracle_mod.REL, eb, leaf_size=cfg.leaf_size)
            else:
                ref, _ = oracle_mod.compress(pos, oracle_mod.REL, eb, leaf_size=cfg.leaf_size)
            if cfg.flags & pc.PC_FLAG_REORDER:
                ref, _, _ = oracle_mod.reorder(ref)
            assert o[:sz].cpu().numpy().tobytes() == ref


def test_batch_reports_failed_items(pc):
    dev = torch.device("cuda:0")
    good = torch.from_numpy(synth.uniform(5000, seed=1)).to(dev)
    outs = [torch.empty(pc.pc_compress_bound(5000, pc.PC_F32), dtype=torch.uint8, device=dev) for _ in range(3)]
    sizes, statuses = pc.pc_compress_batch([(good, pc.PC_EB_REL, 1e-3, 0), (good, pc.PC_EB_REL, 0.0, 0),
                                            (good, pc.PC_EB_ABS, 1e-2, 0)], outs, lanes=2)
    assert statuses[0] == pc.PC_OK and statuses[2] == pc.PC_OK
    assert statuses[1] == pc.PC_ERR_ARG and sizes[1] == 0
    assert torch.equal(outs[0][:sizes[0]], _alone(pc, good, pc.PC_EB_REL, 1e-3, 0))


def test_decompress_batch_kinds_and_failures(pc, oracle_mod):
    """One batched decompression over streams of every kind (float32, float64,
    lossless axes, empty) and broken items (a corrupt leaf record, a truncated
    stream, an output too small, an output 4 bytes off 16-byte alignment): each
    item's status and output equal the plain call's, and the decoded floats the
    oracle's."""
    dev = torch.device("cuda:0")
    specs = [("cosmology", 70_000, np.float32, pc.PC_EB_REL, 1e-3), ("fluid", 50_000, np.float64, pc.PC_EB_ABS, 1e-4),
             ("cosmology", 30_000, np.float32, pc.PC_EB_REL, 1e-9), ("uniform", 0, np.float32, pc.PC_EB_REL, 1e-3),
             ("uniform", 90_001, np.float32, pc.PC_EB_REL, 1e-2), ("fluid", 20_000, np.float64, pc.PC_EB_REL, 1e-12)]
    pos, streams = [], []
    for gen, n, dt, m, eb in specs:
        p = synth.by_name(gen, n, seed=n % 13, dtype=dt) if n else np.zeros((0, 3), dt)
        d = torch.from_numpy(p).to(dev)
        c = pc.Compressor(max(n, 1), pc.PC_F32 if dt == np.float32 else pc.PC_F64, device=dev)
        size = c.compress(d, m, eb)
        om = oracle_mod.REL if m == pc.PC_EB_REL else oracle_mod.ABS
        ref, _ = oracle_mod.compress(p, om, eb)
        assert c.out[:size].cpu().numpy().tobytes() == ref
        pos.append(p)
        streams.append(c.out[:size].clone())
    # broken items: a corrupt leaf record (its zero byte set), a truncated stream, too small an output
    bad = streams[0].clone()
    bad[96 + 32 * 2 + 31] = 1
    items = [(s, s.numel(), torch.empty(p.shape, dtype=torch.from_numpy(p).dtype, device=dev))
             for s, p in zip(streams, pos)]
    items.append((bad, bad.numel(), torch.empty(pos[0].shape, dtype=torch.float32, device=dev)))
    items.append((streams[1], streams[1].numel() - 4, torch.empty(pos[1].shape, dtype=torch.float64, device=dev)))
    items.append((streams[4], streams[4].numel(), torch.empty((10, 3), dtype=torch.float32, device=dev)))
    # an output 4 bytes off 16-byte alignment: the float32 streams then decode without 16-byte stores
    off = torch.empty(pos[4].size + 1, dtype=torch.float32, device=dev)[1:].view(-1, 3)
    items.append((streams[4], streams[4].numel(), off))
    outs = [o for _, _, o in items]
    got = pc.pc_decompress_batch([s for s, _, _ in items], [nb for _, nb, _ in items], outs)
    for (s, nb, o), st in zip(items, got):
        alone = torch.zeros_like(o)
        c = pc.Compressor(max(o.shape[0], 1), pc.PC_F32 if o.dtype == torch.float32 else pc.PC_F64, device=dev)
        try:
            c.decompress(s[:nb] if nb <= s.numel() else s, alone, nb)
            want = pc.PC_OK
        except pc.PCError as e:
            want = e.status
        assert st == want
        if st == pc.PC_OK and o.shape[0]:
            assert torch.equal(o, alone)
    expect = [pc.PC_OK] * 6 + [pc.PC_ERR_CORRUPT, pc.PC_ERR_CORRUPT, pc.PC_ERR_CAPACITY, pc.PC_OK]
    assert got == expect
    for p, s, o in zip(pos, streams, outs[:6]):
        if p.shape[0]:
            assert o.cpu().numpy().tobytes() == oracle_mod.decompress(s.cpu().numpy().tobytes()).tobytes()
    assert torch.equal(outs[9], outs[4])


@pytest.mark.parametrize("arena_mb,lanes", [(1024, 4), (96, 3)])
def test_server_mix_equals_alone(pc, arena_mb, lanes):
    """Compress requests, then decompress requests of their streams, submitted
    together; with a small arena they wait for room and still all finish."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(7)
    snaps = []
    for i in range(18):
        n = int(round(10 ** rng.uniform(3, 5.5)))
        snaps.append(torch.from_numpy(synth.cosmology(n, seed=100 + i)).to(dev))
    ebs = [float(rng.choice([1e-3, 1e-4])) for _ in snaps]
    alone = [_alone(pc, p, pc.PC_EB_REL, eb, 0) for p, eb in zip(snaps, ebs)]
    arena = torch.empty(arena_mb << 20, dtype=torch.uint8, device=dev)
    srv = pc.Server(arena, lanes=lanes)
    try:
        for i, (p, eb) in enumerate(zip(snaps, ebs)):
            srv.submit_compress(p, pc.PC_EB_REL, eb, tag=i)
        # decompress requests of the alone streams, in the same mix
        for i, a in enumerate(alone):
            srv.submit_decompress(a, a.numel(), snaps[i].shape[0], pc.PC_F32, tag=1000 + i)
        got = {}
        while len(got) < 2 * len(snaps):
            for c in srv.poll(wait=True):
                assert c.status == pc.PC_OK, (c.tag, c.status)
                assert c.t_submit <= c.t_start <= c.t_done
                if c.tag < 1000:
                    got[c.tag] = srv.output(c).clone()
                else:
                    got[c.tag] = srv.output(c, torch.float32).clone()
                srv.release(c)
        for i, a in enumerate(alone):
            assert torch.equal(got[i], a)
            ref = torch.empty_like(snaps[i])
            pc.Compressor(snaps[i].shape[0], pc.PC_F32, device=dev).decompress(a, ref, a.numel())
            assert torch.equal(got[1000 + i], ref)
        pending, in_use = srv.stats()
        assert pending == 0 and in_use == 0
    finally:
        srv.close()


def test_server_rejects_what_never_fits(pc):
    dev = torch.device("cuda:0")
    arena = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    srv = pc.Server(arena, lanes=2)
    try:
        big = torch.from_numpy(synth.uniform(200_000, seed=2)).to(dev)
        small = torch.from_numpy(synth.uniform(100, seed=3)).to(dev)
        srv.submit_compress(big, pc.PC_EB_REL, 1e-3, tag=1)
        srv.submit_compress(small, pc.PC_EB_REL, 1e-3, tag=2)
        done = {}
        while len(done) < 2:
            for c in srv.poll(wait=True):
                done[c.tag] = c.status
                if c.status == pc.PC_OK:
                    srv.release(c)
        assert done == {1: pc.PC_ERR_CAPACITY, 2: pc.PC_OK}
    finally:
        srv.close()
