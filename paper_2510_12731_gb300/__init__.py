"""GB300-native wFQ / wFQFmu plasmonic linear-response solver."""
