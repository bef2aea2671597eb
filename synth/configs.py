"""The five synthetic workloads, as plain numbers.

Shapes follow the paper's benchmark (Sec. 5.2: HTRU-like band, 1024
channels of 2-bit samples at 64 us, 1196 trials over 0 <= DM < 1000) and a
tiny case small enough for the CPU oracle.  Trial-DM lists that follow the
bounded-smearing rule are NOT computed here (that is method arithmetic);
entries give the rule's parameters instead.
"""

TINY = dict(
    name="tiny-64ch-u8",
    nchans=64, f0=1500.0, df=-1.0, dt=64e-6, nbits=8,
    dms=dict(kind="linear", lo=0.0, step=1.0, n=101),
    nsamps=16384, seed=1,
    noise=dict(kind="normal_u8", mean=128.0, sd=16.0),
    pulses=[dict(dm_index=50, t0=8000, width=4, amp=40)],
)

SURVEY = dict(
    name="survey-1024ch-u2",
    nchans=1024, f0=1581.8, df=-0.390625, dt=64e-6, nbits=2,
    dms=dict(kind="rule", lo=0.0, hi=1000.0, width_us=40.0, tol=1.25),
    nsamps=1 << 19, seed=1,
    noise=dict(kind="uniform"),
    pulses=[dict(dm=120.0, t0=100000, width=8, value=3),
            dict(dm=560.0, t0=250000, width=8, value=3),
            dict(dm=940.0, t0=400000, width=8, value=3)],
)

FORMAT_SWEEP = dict(
    name="format-sweep-1024ch",
    nchans=1024, f0=1581.8, df=-0.390625, dt=64e-6,
    nbits_list=(1, 4, 8, 32),
    dms=dict(kind="rule", lo=0.0, hi=2000.0, width_us=40.0, tol=1.25),
    nsamps_list=(1 << 17, 1 << 20), seed=3,
)

SUBBAND = dict(
    name="subband-1024ch-u2-32x32",
    nchans=1024, f0=1581.8, df=-0.390625, dt=64e-6, nbits=2,
    dms=dict(kind="rule", lo=0.0, hi=1000.0, width_us=40.0, tol=1.25),
    nsamps=1 << 19, seed=1, chans_per_subband=32, dms_per_nominal=32,
)

SERVING = dict(
    name="serving-13beam-u8",
    nbeams=13, nbits=8, dt=64e-6,
    bands=[dict(nchans=512, f0=1581.8, df=-0.78125),
           dict(nchans=1024, f0=1581.8, df=-0.390625)],
    dms=dict(kind="rule", lo=0.0, hi=2000.0, width_us=40.0, tol=1.25),
    gulp_lo=1 << 16, gulp_hi=1 << 19, seed=5, offered_load=0.7,
)

ALL = [TINY, SURVEY, FORMAT_SWEEP, SUBBAND, SERVING]


def linear_dms(spec):
    """Trial DMs of a ``linear`` spec (plain arithmetic progression)."""
    return [spec["lo"] + i * spec["step"] for i in range(spec["n"])]
